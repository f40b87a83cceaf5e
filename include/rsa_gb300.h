/*
 * rsa_gb300.h -- C ABI of the GB300 (sm_103a) batched RSA modular
 * exponentiation library (librsagpu.so).
 *
 * The operation (paper "Analysis of RSA Algorithm using GPU Programming",
 * Sec. 2 and Sec. 3.2-3.3, and the decryption note of Sec. 11):
 *     encryption  C = M^e mod n
 *     decryption  M = C^d mod n
 * with 0 <= M < n, n = p*q (key generation, Fig. 1).  Decryption can run
 * through the Chinese remainder theorem (p and q supplied at key load), which
 * gives the same value as C^d mod n for any d >= 1.
 *
 * Conventions for every entry point:
 *   - Big numbers are arrays of 32-bit limbs, little-endian by limb (limb 0 is
 *     the least significant); bytes inside a limb are in the machine's order.
 *   - A key of nbits bits has L = nbits/32 limbs; its message and result rows
 *     have exactly L limbs.  p and q have L/2 limbs each.
 *   - "device pointer" arguments must point to memory of the context's device
 *     (cudaMalloc'd or a PyTorch CUDA tensor); "host pointer" arguments to
 *     ordinary host memory.  The caller owns every buffer it passes; the
 *     library owns its key table and workspace, which count against the
 *     memory budget given at context creation.
 *   - Calls taking a stream (a cudaStream_t passed as void*, NULL = legacy
 *     default stream) only enqueue work and return; nothing is implicitly
 *     synchronised.  rsa_sync() waits for the stream and reports device-side
 *     errors recorded since the previous rsa_sync().
 *   - Return value: RSA_OK (0) or a negative rsa_status.  The message of the
 *     most recent failure on the calling thread is in rsa_last_error().
 *   - One context may be used from several host threads; calls are serialised
 *     internally.
 */
#ifndef RSA_GB300_H
#define RSA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsa_ctx rsa_ctx; /* opaque, library-owned */

typedef enum rsa_status {
    RSA_OK = 0,
    RSA_ERR_ARG = -1,         /* null pointer, bad enum, count out of range */
    RSA_ERR_KEY = -2,         /* even modulus, p*q != n, zero exponent, unknown/unloaded key id,
                                 private operation on a key loaded without d (or without p, q) */
    RSA_ERR_RANGE = -3,       /* per operation: message >= n (its output row is zeroed) */
    RSA_ERR_NOMEM = -4,       /* memory budget exceeded or device allocation failed */
    RSA_ERR_CUDA = -5,        /* a CUDA runtime call failed */
    RSA_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up */
    RSA_ERR_UNSUPPORTED = -7, /* key size or operation kind not supported */
    RSA_ERR_VERIFY = -8       /* per operation of rsa_verify_key: s^e mod n differs from the
                                 expected representative */
} rsa_status;

/* Which exponent an operation uses. */
typedef enum rsa_exp_sel {
    RSA_EXP_PUBLIC = 0,        /* x = e, variable-time binary method (e is public), Fig. 5 */
    RSA_EXP_PRIVATE_CRT = 1,   /* x = d via p, q: two half-size constant-time fixed-window
                                  exponentiations (Fig. 6 digits) and Garner recombination */
    RSA_EXP_PRIVATE_PLAIN = 2  /* x = d directly mod n, constant-time fixed window */
} rsa_exp_sel;

/* Supported key sizes: nbits in {1024, 2048, 3072, 4096} (multi-limb path), and
 * nbits = 32 for moduli below 2^32 (single-limb path of the paper's toy example,
 * n = 17947, e = 131, d = 137, Sec. 2).  PRIVATE_CRT needs p and q; 3072/4096-bit
 * PUBLIC and PRIVATE_PLAIN run with four lanes per operation by default. */

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the library's
 * own device memory (key table + workspace); 0 selects 2 GiB.  *out receives the
 * context.  Errors: RSA_ERR_ARG, RSA_ERR_CUDA. */
int rsa_ctx_create(rsa_ctx **out, int device, size_t mem_budget_bytes);

/* Release every key and all workspace.  Waits for work the library enqueued. */
int rsa_ctx_destroy(rsa_ctx *ctx);

/* Load a key (paper Fig. 1: public key (e, n), private key d, primes p, q).
 * All pointers are host pointers and are copied; the library precomputes the
 * per-key Montgomery constants (n' = -n^-1 mod 2^32, R mod n, R^2 mod n with
 * R = 2^(32*L); for p and q also R^2, R^3 mod p|q, dp = d mod (p-1),
 * dq = d mod (q-1), qinv = q^-1 mod p) and keeps them resident on the device.
 *   n       L = nbits/32 limbs, odd, top limb nonzero for nbits >= 1024
 *   e       e_limbs limbs (1 <= e_limbs <= L), e >= 1
 *   d       L limbs or NULL (then only RSA_EXP_PUBLIC is allowed), d >= 1
 *   p, q    L/2 limbs each, or both NULL (then RSA_EXP_PRIVATE_CRT is refused);
 *           must be odd with p*q == n and gcd(p, q) == 1
 * *key_id_out receives a small non-negative id.
 * Errors: RSA_ERR_ARG, RSA_ERR_KEY, RSA_ERR_UNSUPPORTED, RSA_ERR_NOMEM, RSA_ERR_CUDA. */
int rsa_keyload(rsa_ctx *ctx, uint32_t nbits, const uint32_t *n, const uint32_t *e,
                uint32_t e_limbs, const uint32_t *d, const uint32_t *p, const uint32_t *q,
                int32_t *key_id_out);

/* Host only, no device needed: compute the key record rsa_keyload() would
 * upload for the same arguments (header, n, R^2 mod n, R mod n, e, d, and for
 * CRT keys p, q, R^2 and R^3 mod p|q, R mod p|q, qinv, dp, dq; the word layout
 * is the one documented in the library's keyrec.h).  With rec == NULL only
 * *rec_words is set.  Same validation and errors as rsa_keyload(), plus
 * RSA_ERR_ARG when rec_capacity_words is too small. */
int rsa_key_record(uint32_t nbits, const uint32_t *n, const uint32_t *e, uint32_t e_limbs,
                   const uint32_t *d, const uint32_t *p, const uint32_t *q, uint32_t *rec,
                   size_t rec_capacity_words, size_t *rec_words);

/* Forget a key; its id may be reused.  Waits for work the library enqueued. */
int rsa_keyunload(rsa_ctx *ctx, int32_t key_id);

/* Query a loaded key: bit size, whether d and whether p, q were supplied. */
int rsa_key_info(rsa_ctx *ctx, int32_t key_id, uint32_t *nbits, int32_t *has_d, int32_t *has_crt);

/* Uniform batch: `count` operations, all under key `key_id` with exponent `exp_sel`.
 *   msgs, out   device pointers to count rows of L limbs (row i at msgs + i*L);
 *               out may equal msgs (in-place) but must not partially overlap it
 *   op_status   device pointer to count int32 (RSA_OK or RSA_ERR_RANGE), or NULL
 * Enqueued on `stream`.  Errors (returned before anything is enqueued):
 * RSA_ERR_ARG, RSA_ERR_KEY, RSA_ERR_UNSUPPORTED, RSA_ERR_NOMEM, RSA_ERR_CUDA. */
int rsa_modexp_key(rsa_ctx *ctx, int32_t key_id, int32_t exp_sel, uint64_t count,
                   const uint32_t *msgs, uint32_t *out, int32_t *op_status, void *stream);

/* Signatures on the same kernels (Sec. 3.2-3.3: signing applies the private
 * exponent, verifying the public one).  A "representative" is the integer to be
 * signed, already hashed and padded by the caller (no hashing or padding here),
 * as L limbs below n.
 *
 * rsa_sign_key: sigs[i] = reps[i]^d mod n, through p, q (CRT) when the key has
 *   them, else with d directly.  reps, sigs: device pointers to count rows of L
 *   limbs (16-byte aligned; sigs may equal reps).  op_status: device pointer to
 *   count int32 (RSA_OK, or RSA_ERR_RANGE for a representative >= n, whose
 *   signature row is zeroed), or NULL.
 * rsa_verify_key: op_status[i] = RSA_OK when sigs[i]^e mod n == reps[i],
 *   RSA_ERR_VERIFY when it differs, RSA_ERR_RANGE when sigs[i] >= n.  sigs,
 *   reps: device pointers to count rows of L limbs; op_status is required (the
 *   verdicts).  Scratch for the recovered representatives comes from the
 *   context's budget.
 * Both are enqueued on `stream`.  Errors (before anything is enqueued):
 * RSA_ERR_ARG, RSA_ERR_KEY (rsa_sign_key on a key loaded without d),
 * RSA_ERR_UNSUPPORTED, RSA_ERR_NOMEM, RSA_ERR_CUDA. */
int rsa_sign_key(rsa_ctx *ctx, int32_t key_id, uint64_t count, const uint32_t *reps, uint32_t *sigs,
                 int32_t *op_status, void *stream);
int rsa_verify_key(rsa_ctx *ctx, int32_t key_id, uint64_t count, const uint32_t *sigs, const uint32_t *reps,
                   int32_t *op_status, void *stream);

/* Batch Miller-Rabin probable-prime tests, the step before key generation
 * (Fig. 1 asks for two large primes; the paper names no test).  Candidate i is
 * the odd integer n_i of nbits/32 limbs at cands + i*L (nbits 512, 1024 or 2048; the
 * top bit need not be set); its `rounds` bases are the rows
 * bases + (i*rounds + r)*L, each in [2, n_i - 2] (drawn by the caller).
 * Writing n_i - 1 = d 2^s with d odd, base a passes when a^d = 1 or
 * a^(d 2^r) = n_i - 1 (mod n_i) for some r < s.  verdicts[i] = 1 when every
 * base passes (probable prime), 0 when some base proves n_i composite, -1 for
 * an even candidate or one below 5.  All pointers are device pointers (rows
 * 16-byte aligned); the powers are constant-time in the candidate.  Enqueued
 * on `stream`.  Errors: RSA_ERR_ARG, RSA_ERR_UNSUPPORTED, RSA_ERR_NOMEM,
 * RSA_ERR_CUDA. */
int rsa_mr_batch(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *cands, uint32_t rounds,
                 const uint32_t *bases, int32_t *verdicts, void *stream);

/* Batch GCD (weak-key detection; the introduction rests RSA's security on the
 * difficulty of factoring n, and two moduli sharing a prime are both factored
 * by one gcd).  For the `count` moduli n_i of nbits/32 limbs at
 * moduli + i*L (nbits 512, 1024 or 2048; a modulus may have leading zero
 * limbs), g_i = gcd(n_i, prod_{j != i, n_j valid} n_j).  A modulus is valid
 * when it is odd and at least 3; invalid ones are left out of every product.
 * gcds (count rows of L limbs, or NULL) receives g_i (zeros for an invalid
 * n_i); flags (count int32, or NULL) receives 0 when g_i = 1 (n_i shares no
 * factor with the others), 1 when 1 < g_i < n_i (g_i is a proper factor),
 * 2 when g_i = n_i (a duplicate modulus, or each prime of n_i is shared:
 * separate it with pairwise gcds), -1 for an invalid n_i.  At least one of
 * gcds and flags must be given.  All pointers are device pointers (rows
 * 16-byte aligned).  The form is the one rsa_batch_gcd_ex picks with
 * RSA_GCD_AUTO.  Enqueued on `stream`.  Errors: RSA_ERR_ARG (null or misaligned
 * pointers, count above 2^26), RSA_ERR_UNSUPPORTED, RSA_ERR_NOMEM,
 * RSA_ERR_CUDA. */
int rsa_batch_gcd(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds,
                  int32_t *flags, void *stream);

/* Forms of the batch GCD; both give the same gcds and flags.
 * RSA_GCD_SCAN: modulus by modulus over block products of the others,
 *   about count^2 / 2 Montgomery-word operations of the modulus size, a few
 *   kernels, little memory.
 * RSA_GCD_TREE: a product tree of the moduli and a remainder tree of
 *   prod n_j modulo every n_i^2 (Montgomery remainders, no divisions), then
 *   (prod n_j / n_i) mod n_i and a binary gcd per modulus: quasi-linear work,
 *   products of long numbers by three-prime number-theoretic transforms.
 *   Needs rsa_batch_gcd_tree_bytes of device memory within the context's
 *   budget (2.7 GiB for 2^17 moduli of 2048 bits, 23 GiB for 2^20) and
 *   count (rounded up to a power of two) x nbits / 32 <= 2^26.
 * RSA_GCD_AUTO: the tree from count x nbits / 32 >= 2^18 (4096 moduli of 2048
 *   bits, 8192 of 1024, 16384 of 512) when it fits (the size limit and the
 *   memory budget), else the scan. */
#define RSA_GCD_AUTO 0
#define RSA_GCD_SCAN 1
#define RSA_GCD_TREE 2
/* rsa_batch_gcd in a given form.  Errors as rsa_batch_gcd, and RSA_ERR_ARG for
 * an unknown method or a tree beyond its size limit; RSA_ERR_NOMEM when the
 * tree's memory exceeds the budget. */
int rsa_batch_gcd_ex(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds,
                     int32_t *flags, int method, void *stream);
/* The form RSA_GCD_AUTO takes for `count` moduli on this context now
 * (RSA_GCD_SCAN or RSA_GCD_TREE).  No GPU work.  Errors as rsa_batch_gcd. */
int rsa_batch_gcd_method(rsa_ctx *ctx, uint32_t nbits, uint64_t count, int *method);
/* Device bytes the tree form takes for `count` moduli of nbits (its levels,
 * transform scratch and twiddle tables).  Errors: RSA_ERR_UNSUPPORTED,
 * RSA_ERR_ARG (null pointer, beyond the size limit). */
int rsa_batch_gcd_tree_bytes(uint32_t nbits, uint64_t count, uint64_t *bytes);
/* rsa_batch_gcd with host buffers: moduli, gcds (or NULL) and flags (or NULL)
 * are host pointers (pinned memory copies fastest); the copies in and out run
 * on `stream`, and the call returns when the results are in host memory.
 * Device buffers come from the context's workspace.  Errors as rsa_batch_gcd. */
int rsa_batch_gcd_host(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds,
                       int32_t *flags, void *stream);
/* The work split rsa_batch_gcd would use for `count` moduli: the block size
 * of its block products (moduli multiplied together before the per-modulus
 * reduction) and the number of parts the moduli range is cut into for load
 * balance (each part's partial products are multiplied in a last kernel).
 * For work accounting; no GPU work.  Errors as rsa_batch_gcd. */
int rsa_batch_gcd_plan(rsa_ctx *ctx, uint32_t nbits, uint64_t count, uint32_t *block, uint64_t *parts);

/* Ragged batch: operation i uses key key_ids[i] (any loaded key, any size) and
 * exponent exp_sel[i]; its message is the L_i limbs at msgs + limb_offsets[i]
 * and its result goes to out + limb_offsets[i].  All five arrays are device
 * pointers of `count` entries (op_status may be NULL).  The library groups the
 * operations on the device by (key, exponent kind), forms tiles of 32, orders
 * the tiles longest-first and runs them in one persistent kernel launch; the
 * launch sequence is captured once into a CUDA graph and replayed.  Operations
 * whose key id is invalid or whose exponent kind the key cannot serve get
 * RSA_ERR_KEY in op_status and a zeroed row; rsa_sync() then also returns
 * RSA_ERR_KEY.  Enqueued on `stream`. */
int rsa_modexp_batch(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids,
                     const uint8_t *exp_sel, const uint64_t *limb_offsets,
                     const uint32_t *msgs, uint32_t *out, int32_t *op_status, void *stream);

/* Host-buffer forms of the two calls above: every pointer is a host pointer.
 * The library copies the inputs to its device workspace, runs the batch on
 * `stream`, copies the results back and waits for completion.  These are the
 * end-to-end entry points (host->device and device->host copies included). */
int rsa_modexp_key_host(rsa_ctx *ctx, int32_t key_id, int32_t exp_sel, uint64_t count,
                        const uint32_t *msgs, uint32_t *out, int32_t *op_status, void *stream);
int rsa_modexp_batch_host(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids,
                          const uint8_t *exp_sel, const uint64_t *limb_offsets,
                          uint64_t total_limbs, const uint32_t *msgs, uint32_t *out,
                          int32_t *op_status, void *stream);

/* CRT decryption that allocates no memory (no context, no cudaMalloc).
 * The paper has no counterpart; this exists for callers that cannot allocate
 * device memory at call time -- code inside a CUDA graph capture, plug-ins whose
 * host process owns all device memory through its own pool, or services that
 * forbid allocation after start-up so a request can never fail on it.
 *   key_record  device pointer to the words rsa_key_record() returns for a key
 *               given with d, p and q (copied by the caller into memory it owns)
 *   nbits       1024, 2048, 3072 or 4096 (other sizes: RSA_ERR_UNSUPPORTED)
 *   msgs, out   device pointers to count rows of nbits/32 limbs (16-byte aligned)
 *   op_status   device pointer to count int32 (RSA_OK / RSA_ERR_RANGE) or NULL
 * Results are identical to rsa_modexp_key(..., RSA_EXP_PRIVATE_CRT, ...).
 * The window-table scratch is a fixed 32 MiB array inside the library, held on
 * every GPU that loads it until the process exits; the launch is sized to fit
 * it (window width 4), so throughput is below rsa_modexp_key's.  All calls
 * share that array: calls that overlap on the GPU race and must be ordered on
 * one stream.  The first call on a device looks up the array's address with
 * that device current; make it before any stream capture.  Only the device's
 * primary context (the CUDA runtime's) is supported: the array's address is
 * cached per device, and a separate driver-API context on the same device
 * holds its own copy of the array.  Enqueued on `stream`; errors are returned
 * before anything is enqueued. */
int rsa_crt_decrypt_noalloc(const uint32_t *key_record, uint32_t nbits, uint64_t count,
                            const uint32_t *msgs, uint32_t *out, int32_t *op_status, void *stream);

/* ---------------------------------------------------------------- serving
 * A request loop on top of rsa_modexp_batch.  A scheduler thread packs
 * requests that have arrived, of one modulus size (any keys and kinds of that
 * size; the oldest waiting request picks the size), into one ragged batch per
 * free slot, and runs up to max_inflight_batches batches at once on separate
 * streams, so requests arriving while others are on the GPU start without
 * waiting for them (continuous batching) and a batch finishes at its own size's
 * latency.  Once the operations in flight fill a wave of the GPU, at most three
 * batches run at once, so waiting requests gather into larger batches.  Admission is by bytes in flight: every batch takes a range of one
 * device arena of mem_budget_bytes (messages, results and per-operation
 * metadata: 8L + 17 bytes per operation, plus alignment), and a batch that does
 * not fit in a free range waits until batches in flight finish and give their
 * ranges back.  Key state stays resident in the context.  Results are copied
 * into each request's host buffer. */
typedef struct rsa_server_cfg {
    int32_t max_inflight_batches; /* concurrent batches (streams); 0 -> 16 */
    int32_t batch_window_us;      /* wait this long after the first arrival for more; 0 -> 200 */
    int32_t max_batch_ops;        /* operations per batch (and per request); 0 -> 65536 */
    int32_t flags;                /* RSA_SERVER_MIX_SIZES: a batch takes requests of every
                                     modulus size (default: one size per batch, see above) */
    uint64_t mem_budget_bytes;    /* device bytes for in-flight requests (one arena, counted
                                     against the context's budget; the loop also pins the same
                                     amount of host memory for staging); 0 -> 2 GiB */
} rsa_server_cfg;
#define RSA_SERVER_MIX_SIZES 1

typedef struct rsa_request {
    int32_t key_id;
    int32_t exp_sel;
    uint32_t count;               /* messages in this request */
    uint32_t reserved;
    const uint32_t *msgs;         /* host: count rows of the key's L limbs */
    uint32_t *out;                /* host: count rows, written when done */
    int32_t *status;              /* host: count statuses, or NULL */
    uint64_t arrive_ns;           /* arrival time, ns after rsa_server_start; 0 = at submit */
} rsa_request;

typedef struct rsa_server_stats {
    uint64_t submitted, completed, rejected, ops_completed, batches;
    uint64_t peak_bytes;          /* largest arena footprint of the batches in flight */
    double p50_us, p99_us, mean_us, max_us;   /* request latency: arrival -> result in host buffer */
    double span_s;                /* first arrival -> last completion */
} rsa_server_stats;

/* Start the request loop of `ctx` (one per context).  The buffers a request
 * points to must stay valid until it completes. */
int rsa_server_start(rsa_ctx *ctx, const rsa_server_cfg *cfg);
/* Queue a request; *ticket identifies it.  A request that fits the budget is
 * never refused for lack of room: it waits for batches in flight.  RSA_ERR_NOMEM
 * when the request alone exceeds the budget (or holds more than max_batch_ops
 * messages), RSA_ERR_KEY / RSA_ERR_ARG for a bad key or kind. */
int rsa_server_submit(rsa_ctx *ctx, const rsa_request *req, uint64_t *ticket);
/* Queue n requests at once (in arrival order); tickets (n entries) may be NULL.
 * Stops at the first refused request and returns its error; *accepted (may be
 * NULL) receives how many were queued. */
int rsa_server_submit_many(rsa_ctx *ctx, const rsa_request *reqs, uint32_t n, uint64_t *tickets,
                           uint32_t *accepted);
/* The loop's arrival clock: nanoseconds since rsa_server_start. */
int rsa_server_clock(rsa_ctx *ctx, uint64_t *ns_since_start);
/* *done = 1 when the request completed, 0 while pending, a negative status on failure. */
int rsa_server_poll(rsa_ctx *ctx, uint64_t ticket, int32_t *done);
/* Wait until every submitted request completed (timeout_ms <= 0: no limit).
 * RSA_ERR_TIMEOUT when the limit passes first. */
int rsa_server_drain(rsa_ctx *ctx, int32_t timeout_ms);
/* Latency and throughput counters since start (or the last reset). */
int rsa_server_get_stats(rsa_ctx *ctx, rsa_server_stats *s, int32_t reset);
/* Stop the loop: requests that have arrived are run to completion; requests
 * whose arrival time is still in the future are cancelled (never run,
 * RSA_ERR_TIMEOUT written to each of their status entries when a status array
 * was given).  Releases the loop's buffers; tickets are invalid afterwards. */
int rsa_server_stop(rsa_ctx *ctx);

/* Wait for `stream` and return the first device-side error recorded since the
 * previous call (RSA_ERR_KEY, RSA_ERR_TIMEOUT), RSA_ERR_CUDA, or RSA_OK. */
int rsa_sync(rsa_ctx *ctx, void *stream);

/* Message of the most recent failure on the calling thread ("" if none). */
const char *rsa_last_error(void);

/* Launch parameters of the multi-limb kernels.  Zero fields mean "automatic". */
typedef struct rsa_tuning {
    int32_t window;        /* fixed-window width w for private exponents, 3..6; for
                              sliding-window public exponents the maximum window */
    int32_t warps_per_cta; /* warps per CTA (even for CRT: warp pairs), 1..8 */
    int32_t ctas_per_sm;   /* resident CTAs per SM the grid is sized for */
    int32_t variant;       /* squarings of private exponents: 1 = through the general
                              CIOS multiply, 2 = separated square + reduction (fewer
                              word products, but a larger instruction footprint; slower
                              on GB300); 3 = RSA-2048, -3072 and -4096 CRT: the
                              Montgomery reduction on the tensor cores (tcgen05 MMAs of
                              byte digits against Toeplitz matrices of p, q and -p^-1,
                              -q^-1; for 1536/2048-bit primes in two rounds of half the
                              prime size; the per-message product stays on the CUDA
                              cores; windows 3 and 4); 0 = automatic: 3 for RSA-2048 CRT
                              (window 3), RSA-3072 CRT batches of at least 8192
                              operations (window 4) and RSA-4096 CRT batches of at least
                              12288 (window 3), 1 otherwise.  For RSA_EXP_PUBLIC (moduli up to 2048
                              bits): 1 = binary method (Fig. 5), 2 = sliding windows
                              of up to `window` bits (Fig. 7; window 4..6, default 5),
                              3 = 2048-bit keys: binary method with the Montgomery
                              reductions mod n on the tensor cores (two rounds of 2^1024,
                              as for an RSA-4096 prime; status RSA_ERR_TIMEOUT if a
                              bounded MMA wait gives up), 0 = automatic: 3 for 2048-bit
                              keys, exponents up to 64 bits and at least 4096 operations,
                              else sliding for exponents longer than 64 bits */
    int32_t threads_per_op; /* lanes cooperating on one operation: 1, 2 or 4 (numbers
                              sliced over the lanes, warp-shuffle carries); 0 = automatic
                              (4 above 2048 bits, else 1).  PRIVATE_PLAIN takes 1 up to
                              2048 bits and 4 above; other combinations without a kernel
                              return RSA_ERR_UNSUPPORTED from the launching call */
    /* The last three fields apply to RSA_TUNE_RAGGED only (0 elsewhere): */
    int32_t window_big;    /* fixed-window width of 3072/4096-bit CRT (4 or 5; 0 = 5) */
    int32_t window_tc;     /* window of the 2048-bit tensor-core group (3 or 4; 0 = 3);
                              the 3072- and 4096-bit groups run windows 4 and 3 */
    int32_t tc_min_ops;    /* a 2048-, 3072- or 4096-bit CRT bucket (one key) of at
                              least this many operations runs on its size's tensor-core
                              group, in tiles of 128 operations (the last one possibly
                              partial), up to four tiles of one key per CTA at 2048
                              bits, two at 3072/4096; 0 = 128 */
} rsa_tuning;

/* Set (or, with NULL, reset to automatic) the launch parameters used for keys of
 * nbits bits and exponent kind exp_sel.  exp_sel = RSA_TUNE_RAGGED (with nbits 0)
 * addresses rsa_modexp_batch and the request loop: ctas_per_sm caps the resident
 * CTAs per SM of its persistent kernels, threads_per_op picks the lanes per
 * operation of 2048/4096-bit CRT (1: one/four lanes, the throughput shapes; 4:
 * four/sixteen lanes, the latency shapes; 0: automatic, the latency shapes while
 * the work fits one wave of the GPU); window is the CRT window of 1024/2048-bit
 * keys (4 or 5; 0 = 4), window_big that of 3072/4096-bit keys, window_tc and
 * tc_min_ops shape the tensor-core groups; variant 3 sends 2048/3072/4096-bit
 * CRT buckets of at least tc_min_ops operations to their tensor-core groups, 1
 * keeps every operation on the CUDA cores, 0 (automatic) uses the groups except
 * in the latency shapes; warps_per_cta does not apply.  Errors: RSA_ERR_ARG for
 * values outside these ranges. */
#define RSA_TUNE_RAGGED 3
int rsa_set_tuning(rsa_ctx *ctx, uint32_t nbits, int32_t exp_sel, const rsa_tuning *t);
/* Read the parameters currently in force for (nbits, exp_sel). */
int rsa_get_tuning(rsa_ctx *ctx, uint32_t nbits, int32_t exp_sel, rsa_tuning *t);

/* Autotuner: time every launch shape (window 3..6 for private kinds, warps
 * per CTA 2/4/8, CTAs per SM 1/2/max, both squaring variants, lanes per operation,
 * and for 2048/3072/4096-bit CRT the tensor-core path at windows 3 and 4) for key_id's
 * size and kind exp_sel on a synthetic batch of `count` operations (the work
 * of these kernels does not depend on the message values), install the
 * fastest with rsa_set_tuning() and append it to the cache file `cache_path`
 * (NULL: $RSA_TUNE_CACHE, else no file).  A cached entry for the same GPU name,
 * SM count, size, kind and batch-size bucket is used without timing.
 * *best receives the chosen parameters, *best_ms its time per batch.
 * Synchronous; allocates scratch from the context's budget. */
int rsa_autotune(rsa_ctx *ctx, int32_t key_id, int32_t exp_sel, uint64_t count, const char *cache_path,
                 rsa_tuning *best, double *best_ms);

/* Autotuner for ragged batches: times the given batch (the arguments of
 * rsa_modexp_batch, device pointers; out receives its results) by coordinate
 * descent over the RSA_TUNE_RAGGED tuning: each field in turn takes each of its
 * values while the others keep their best so far -- the lanes-per-operation
 * policy (threads_per_op 1, 4), the tensor-core groups (variant 0 automatic,
 * 1 off, 3 on), the smallest CRT bucket they take (tc_min_ops 128, 512) and the
 * 2048-bit group's window (window_tc 3, 4), the CRT windows of 1024/2048-bit
 * (window 4, 5) and 3072/4096-bit keys (window_big 5, 4), and the resident-CTA
 * cap of the CUDA-core groups (ctas_per_sm 0 = occupancy maximum, 2, 4).  A
 * candidate's time is the median of three runs after a warm-up, and its
 * results must equal the first candidate's (a digest of every output row) or
 * it is not taken.  Installs the fastest as the RSA_TUNE_RAGGED tuning and
 * returns it in *best (*best_ms: time per batch).  Synchronous, on a private
 * stream.  Errors: RSA_ERR_ARG, RSA_ERR_KEY (the batch holds operations its
 * keys cannot serve), RSA_ERR_NOMEM, RSA_ERR_CUDA (also when candidates
 * disagree). */
int rsa_autotune_batch(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel,
                       const uint64_t *limb_offsets, const uint32_t *msgs, uint32_t *out, rsa_tuning *best,
                       double *best_ms);

/* Tensor-core operands of one 1024-bit prime m (variant 3), exactly as built at
 * key load: two K-major fp16 matrices in the no-swizzle core-matrix layout
 * ([k/8][row/8][row%8][k%8]), K = 144 (128 byte digits + a 16-column bias block
 * of the value 2048):
 *   bytes [0, 36864):     128 rows, row n, column k < 128: byte n-k of -m^-1 mod 2^1024
 *   bytes [36864, 73728): 128 rows, row j, column k < 128: byte 124+j-k of m
 * (0 where the byte index is outside 0..127).  m: 32 limbs, little-endian, odd.
 * out: host buffer of at least RSA_TC_IMAGE_BYTES bytes.  No GPU is used.
 * Errors: RSA_ERR_ARG (null pointer, short buffer, even m). */
#define RSA_TC_IMAGE_BYTES 73728
int rsa_tc_operand_image(const uint32_t *m, void *out, size_t out_bytes);

/* The same for one prime m of an RSA-3072 or RSA-4096 key (prime_bits 1536 or
 * 2048; variant 3 at those sizes): the Montgomery reduction mod m, R = 2^prime_bits,
 * runs in two rounds of r = 2^(prime_bits/2), each a product by -m^-1 mod r and
 * one by m.  With D = prime_bits/16 byte digits per round and K = D + 16:
 *   bytes [0, 2 D K):       D rows, row n, column k < D: byte n-k of -m^-1 mod r
 *   bytes [2 D K, 6 D K):   2D rows, row j, column k < D: byte D-4+j-k of m
 *   columns D .. D+15 of both: the bias value 2048
 * (0 where the byte index is outside 0 .. D-1, resp. 0 .. 2D-1), in the K-major
 * core-matrix layout above.  m: prime_bits/32 limbs, little-endian, odd.  out:
 * host buffer of at least RSA_TC_ROUND_IMAGE_BYTES(prime_bits) bytes (110592
 * for 2048-bit primes, 64512 for 1536-bit ones).  No GPU is used.  Errors:
 * RSA_ERR_ARG (null pointer, other sizes, short buffer, even m). */
#define RSA_TC_ROUND_IMAGE_BYTES(prime_bits) (6u * ((prime_bits) / 16u) * ((prime_bits) / 16u + 16u))
int rsa_tc_round_operand_image(uint32_t prime_bits, const uint32_t *m, void *out, size_t out_bytes);

/* Counters since context creation. */
typedef struct rsa_stats {
    uint64_t kernel_launches;  /* kernels the library launched (graph replays count their kernels) */
    uint64_t graph_launches;   /* CUDA graph replays */
    uint64_t ops;              /* operations submitted */
    uint64_t bytes_resident;   /* device bytes held against the budget */
} rsa_stats;
int rsa_get_stats(rsa_ctx *ctx, rsa_stats *s);

/* Word products (32x32->64 multiplies) one operation costs under the counting
 * rule 2L^2 + L per Montgomery multiplication on L limbs (operand-scanning
 * CIOS, squarings counted as multiplications), for a key of nbits bits and
 * exponent kind exp_sel: public exponents of e_bits bits with e_weight set
 * bits (binary method), private ones at window width `window` (0 = 5).
 * The figure behind the roofline numbers; it does not depend on the data. */
double rsa_products_per_op(uint32_t nbits, int32_t exp_sel, uint32_t e_bits, uint32_t e_weight,
                           int32_t window);

/* Integer-multiply throughput probe on `device`: *imad_lanes_per_s receives
 * 32-bit multiply-add lane-operations per second from independent mad.lo/
 * mad.hi chains; *chain_products_per_s the 32x32->64 word products per second
 * of mad.lo.cc / madc.hi.cc carry chains shaped like the kernels' product scans
 * (rows of 32 products whose multipliers do not wait for the previous row's
 * last carry), the faster of two occupancies. */
int rsa_imad_probe(int device, double *imad_lanes_per_s, double *chain_products_per_s);

#ifdef __cplusplus
}
#endif
#endif /* RSA_GB300_H */
