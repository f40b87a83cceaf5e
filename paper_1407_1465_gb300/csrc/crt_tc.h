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

// Workspace sizes for a launch of `count` operations on `grid` CTAs.
size_t tc_tables_bytes(int grid, int window);
size_t tc_halves_bytes(uint32_t count);
int tc_grid(uint32_t count, int sm_count);
size_t tc_smem_bytes();

#if defined(__CUDACC__)
// Enqueues the two-prime exponentiation kernel and the recombination kernel.
// wait_polls bounds every wait on an MMA's completion (kDefaultWaitPolls in
// normal use); a tile whose wait gives up reports RSA_ERR_TIMEOUT for its
// operations.
constexpr uint32_t kDefaultWaitPolls = 1u << 22;
cudaError_t launch_crt_tc(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                          int32_t *status, uint32_t count, int grid, int window, void *tables, void *halves,
                          uint32_t wait_polls, cudaStream_t s);
#endif

}  // namespace tcr
}  // namespace rsagpu
