// crt_tc.h -- RSA-2048 CRT decryption with the Montgomery reduction on the
// tensor cores (host-side interface of crt_tc.cu and tcprep.cpp).
#pragma once
#include <cstddef>
#include <cstdint>

namespace rsagpu {
namespace tcr {

constexpr int kH = 32;                   // limbs per prime (1024-bit primes)
constexpr int kDig = 4 * kH;             // byte digits per prime
constexpr int kRows = 128;               // operations per tile (MMA M)
constexpr int kTiles = 4;                // tiles per CTA
constexpr int kThreads = kRows * kTiles; // one thread per operation
constexpr int kN1 = kDig;                // MMA 1 output columns (digits of m)
constexpr int kN2 = kDig;                // MMA 2 output columns (positions 124 .. 251)
constexpr int kN2First = kDig - 4;       // first position MMA 2 produces
constexpr int kKt = kDig + 16;           // K extent of the B images (digits + bias block)
constexpr size_t kImgBm = (size_t)kN1 * kKt * 2;   // 36864 bytes
constexpr size_t kImgBp = (size_t)kN2 * kKt * 2;   // 36864 bytes
constexpr size_t kImgPrime = kImgBm + kImgBp;      // per prime
constexpr size_t kImgKey = 2 * kImgPrime;          // q image, then p image

// Host: the two B operands of one prime m (kH limbs, odd) in the core-matrix
// layout the kernel copies into shared memory.  Returns false if m is even.
bool build_tc_image(const uint32_t *m, uint8_t *out);
// host helpers of the operand builders (tcprep.cpp)
uint16_t f16_of_int(uint32_t x);
size_t core_off(int row, int k, int rows);
uint32_t byte_of(const uint32_t *w, int i);
void neg_inverse_lo(const uint32_t *m, uint32_t *out, int n);   // -m^-1 mod 2^(32 n)

// Workspace sizes for a launch of `count` operations on `grid` CTAs.
size_t tc_tables_bytes(int grid, int window);
size_t tc_halves_bytes(uint32_t count);
int tc_grid(uint32_t count, int sm_count);
size_t tc_smem_bytes();

// Ragged batches: the tensor-core group takes the 128-operation tiles of
// CRT buckets, grouped into chunks of up to kTiles tiles of one key (one CTA
// runs a chunk's tiles side by side, one prime at a time).  The planner writes
// the chunk list; the operations of a chunk are the entries op_start ..
// op_start + nops - 1 of the batch's sorted operation list, 128 per tile, the
// last tile of a bucket possibly partial (its rows past nops compute on the
// chunk's first operation and store nothing).
struct TcChunk {
  const uint32_t *keyrec;   // device key record (keyrec.h)
  const void *image;        // the key's tensor-core operands (q image, then p image)
  int32_t op_start;         // first position in the sorted list
  int32_t ntiles;           // 1 .. kTiles tiles
  int32_t nops;             // operations: 128 (ntiles - 1) < nops <= 128 ntiles
  int32_t pad_;
};
// control words of the ragged tensor-core group inside the batch's control
// block (words 0-15: the planner's ranges and counters, 30-31: the ragged
// autotuner's result digest)
constexpr int kCtlTcChunks = 16;   // chunks planned
constexpr int kCtlTcNext = 17;     // work-item counter of the exponentiation kernel (2 items per chunk)
constexpr int kCtlWords = 32;      // size of the control block in words

#if defined(__CUDACC__)
// Enqueues the two-prime exponentiation kernel and the recombination kernel.
// wait_polls bounds every wait on an MMA's completion (kDefaultWaitPolls in
// normal use); a tile whose wait gives up reports RSA_ERR_TIMEOUT for its
// operations.
constexpr uint32_t kDefaultWaitPolls = 1u << 22;
cudaError_t launch_crt_tc(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                          int32_t *status, uint32_t count, int grid, int window, void *tables, void *halves,
                          uint32_t wait_polls, cudaStream_t s);

// Arguments of the ragged tensor-core kernels (one struct for both, so the
// batch graph passes the same parameter block to each).
struct RaggedTcArgs {
  const TcChunk *chunks;
  uint32_t *ctl;                // control block (kCtlTc* words; error bits in word 2)
  const int32_t *sorted;        // batch position -> operation index
  const uint64_t *offsets;      // operation -> limb offset of its row
  const uint32_t *msgs;
  uint32_t *out;
  int32_t *status;
  void *tables;                 // tc_tables_bytes(grid, window)
  void *halves;                 // tc_halves_bytes(count), indexed by sorted position
  uint32_t count, wait_polls;
  uint32_t ctl_word;            // the group's chunk count in ctl[ctl_word], its work-item counter in ctl[ctl_word + 1]
};
// kernel entry points for the batch graph (window 3 or 4)
const void *ragged_tc_half_fn(int window);
const void *ragged_tc_garner_fn();
constexpr int kRaggedGarnerThreads = 128;
size_t ragged_tc_garner_smem();
#endif

}  // namespace tcr

// RSA-3072 and RSA-4096 CRT with the Montgomery reduction on the tensor cores
// (crt_tc4.cu): primes of H = 48 or 64 limbs, two reduction rounds of
// r = 2^(16H) per Montgomery product, D = 2H byte digits per round.
namespace tc4 {
constexpr int kRows = 128;               // operations per tile (MMA M)
constexpr int kTiles = 2;                // tiles per CTA
constexpr int kThreads = kRows * kTiles;
// B1: D rows (digits of mu) x (D + 16) (digits + bias block); B2: 2D rows
// (positions D-4 .. 3D-5 of mu * m) x (D + 16); fp16
constexpr size_t img_b1_bytes(int H) { return (size_t)(2 * H) * (2 * H + 16) * 2; }
constexpr size_t img_b2_bytes(int H) { return (size_t)(4 * H) * (2 * H + 16) * 2; }
constexpr size_t img_prime_bytes(int H) { return img_b1_bytes(H) + img_b2_bytes(H); }   // 110592 at H = 64
constexpr size_t img_key_bytes(int H) { return 2 * img_prime_bytes(H); }                 // q image, then p image
constexpr bool supported(int H) { return H == 48 || H == 64; }

// Host: the two B operands of one prime m of H limbs (odd): B1 = the Toeplitz
// matrix of -m^-1 mod 2^(16H), B2 = that of m for output positions
// D-4 .. 3D-5, each with the bias block.  Returns false if m is even or H is
// not 48 or 64.
bool build_tc4_image(const uint32_t *m, int H, uint8_t *out);
size_t tc4_tables_bytes(int H, int grid, int window);
size_t tc4_halves_bytes(int H, uint32_t count);
int tc4_grid(uint32_t count, int sm_count);
#if defined(__CUDACC__)
cudaError_t launch_crt_tc4(int H, const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                           int32_t *status, uint32_t count, int grid, int window, void *tables, void *halves,
                           uint32_t wait_polls, cudaStream_t s);
// the public exponent of 2048-bit keys: x^e mod n with n's operands (build_tc4_image(n, kPubH));
// rows of kPubH limbs; status -3 for x >= n (result zeroed), -6 when a bounded MMA wait gave up
constexpr int kPubH = 64;
int pub_tc4_grid(uint32_t count, int sm_count);
size_t pub_tc4_tables_bytes(int grid);
cudaError_t launch_pub_tc4(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                           int32_t *status, uint32_t count, int grid, void *tables, uint32_t wait_polls,
                           cudaStream_t s);
// kernel entry points for the ragged batch graph (tcr::RaggedTcArgs, chunks of up to kTiles tiles)
const void *ragged_tc4_half_fn(int H, int window);
const void *ragged_tc4_garner_fn(int H);
size_t tc4_smem_bytes(int H);
size_t ragged_tc4_garner_smem(int H);
#endif
}  // namespace tc4
}  // namespace rsagpu
