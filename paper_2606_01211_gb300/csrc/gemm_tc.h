// gemm_tc.h -- the batched Encrypt product on the tcgen05 tensor cores.
// Internal to liblwe.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Operand B of the GEMM: the columns of [A | B] (A: n x n from the seed,
// B: n x 8 of the public key) split into two signed 8-bit limbs,
// x = lo + 256 hi (mod 2^16), stored as bf16, K-major: limbs[l][c][i].
struct GemmLimbArgs {
  const uint16_t *A;      // stored A (n x n) or NULL
  const uint8_t *seedA;   // fused: 16-byte seed (device)
  const uint8_t *B;       // n x 8 uint16 (public key matrix) or NULL
  uint32_t n, logq;
  uint16_t *limbs;        // bf16 bits, [2][ncols][n], ncols = n (+8 with B)
};

struct GemmSaArgs {
  const uint16_t *S;      // bf16 bits, [rows][n] (stacked S', K-major)
  const uint16_t *limbs;  // bf16 bits, [2][ncols][n]
  const int8_t *E;        // [rows][n] int8 (E'), nullable
  const int8_t *Epp;      // [rows/8][8][8] int8 (E''), for columns >= n
  const uint8_t *mu;      // 32-byte message slot per item (rows/8 items)
  uint8_t *out;           // item e at out + e * out_stride: rows k of n
                          // uint16 (B'), then C (8 x 8 uint16) at +16 n
  uint64_t out_stride;
  uint32_t *flags;        // compare mode: atomicOr(flags[e], 1) on mismatch
  uint32_t *dev_err;      // bounded waits that run out set bit 0
  uint32_t n;             // K and the A column count
  uint32_t ncols;         // n or n + 8
  uint32_t rows;          // 8 * items
  uint32_t logq, B;
  int cmp;                // 0: write out; 1: compare with out
  int bn;                 // output columns per tile: 64 or 128
  int pair;               // 1: CTA-pair kernel (256 x 128 tiles, cta_group::2)
  uint32_t group_m;       // tile order: M-blocks per group, M fastest inside
                          // a group (0 or 1: row-major tiles)
  // K-split: this launch contracts K = [k0, k0 + 64 * kblocks) only.  The
  // partial sum of earlier passes (mod 2^16, [rows][ncols]) is added from
  // partial_in when set; a non-final pass writes its running sum to
  // partial_out instead of the output (the noise and message are added by
  // the final pass only).
  uint32_t k0, kblocks;
  const uint16_t *partial_in;
  uint16_t *partial_out;
  uint32_t kchunk;        // host: maximum exact K per pass (multiple of 64)
  uint32_t clip;          // |S'| bound c
  uint32_t fast_fold;     // set per pass: every partial sum is below 2^22
  // Odd modulus (the paper's own profile, Tab. 1) when oddq_q != 0: the
  // folded sums are reduced mod oddq_q (Barrett, oddq_m = floor(2^32 / q)),
  // out holds rows of n uint32 (U^T, 256 rows per item), the K-split
  // running sums are uint32 mod q (partial_in / partial_out reinterpreted),
  // and there are no V columns.
  uint32_t oddq_q, oddq_m;
};

cudaError_t lwe_gemm_setup();
bool lwe_gemm_supported(uint32_t n, uint32_t logq, uint32_t clip);
// largest K (multiple of 64) whose partial sums stay below 2^24 for this clip
uint32_t lwe_gemm_kchunk(uint32_t clip);
// number of K passes for (n, clip)
uint32_t lwe_gemm_passes(uint32_t n, uint32_t clip);
int launch_gemm_sa(const GemmSaArgs &a, int num_sms, cudaStream_t st);
void launch_gemm_limbs(const GemmLimbArgs &a, int num_sms, cudaStream_t st);
void launch_s_to_bf16(const int8_t *S, uint64_t count, uint16_t *out, int num_sms,
                      cudaStream_t st);
void launch_selftest_wait(uint32_t *dev_err, uint64_t limit_ns, cudaStream_t st);
// bounds-checked build: skipped accesses of the GEMM kernels (read and clear)
cudaError_t lwe_bounds_read_gemm(unsigned long long *count, unsigned *site);
