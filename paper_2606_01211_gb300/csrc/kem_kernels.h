// kem_kernels.h -- argument blocks and launch wrappers of the KEM kernels.
// Internal to liblwe.so; the public boundary is include/lwe.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Long inputs (pk, c) are hashed as SHA3-256 of the concatenated SHA3-256
// digests of their 1024-byte chunks (a fixed-shape two-level tree).
#define LWE_TREE_CHUNK 1024

enum { NOISE_I8 = 0, NOISE_BF16 = 1 };

// Noise streams are cut into runs of NOISE_RUN consecutive counter blocks;
// one warp generates one run (4 blocks per lane), so one item's round keys
// serve a whole warp and the stores of a warp are contiguous.
#define NOISE_RUN 128
static_assert(256 % NOISE_RUN == 0, "a noise run lies inside one 256-block counter window");

struct NoiseOut {
  void *base;            // item e writes at base + e * item_stride (bytes)
  uint64_t item_stride;  // bytes
  uint32_t nsamples;     // samples per item, sample k from word k%8 of block k/8
  uint32_t domain;       // counter-block domain
  uint32_t fmt;          // NOISE_I8 or NOISE_BF16
  uint32_t runs;         // ceil(ceil(nsamples / 8) / NOISE_RUN)
};

struct NoiseArgs {
  const uint32_t *rk;    // item e: 44 expanded AES round-key words at rk + 44 e
  uint32_t count;
  uint32_t nout;
  uint32_t runs_per_item;
  uint32_t pad0, pad1, pad2;
  NoiseOut out[3];
  uint32_t T[16];        // CDF table, entries >= clip set to 0x7FFF
  const uint4 *tab_img;  // the sampler table for T as k_noise_table writes it
                         // (64 KB, byte w: the sample of word w), or NULL:
                         // each CTA then builds it from T
};

struct MulAsArgs {
  const uint16_t *A;     // stored mode: A of item e at A + e * a_stride
  uint64_t a_stride;     // elements
  const uint8_t *seeds;  // fused mode: seedA of item e at seeds + e*seed_stride
  uint32_t seed_stride;
  uint32_t n;
  uint32_t logq;
  uint32_t row0;         // first row of A computed (A / E / out start at it)
  uint32_t rows;         // rows computed (0 = n)
  uint32_t pad;
  const int8_t *St;      // S^T (8 x n) of item e at St + e * st_stride
  uint64_t st_stride;
  const int8_t *E;       // nullable, n x 8 of item e at E + e * e_stride
  uint64_t e_stride;
  uint8_t *out;          // row i (8 uint16) at out + e*out_stride + 16 i
  uint64_t out_stride;
  uint8_t *out2;         // nullable second copy
  uint64_t out2_stride;
};

struct DecryptArgs {
  const uint8_t *ct;     // item e at ct + e * ct_bytes
  uint64_t ct_bytes;
  const int8_t *St;      // one secret S^T (8 x n)
  const uint8_t *const *sk_ptrs;  // per-item secret keys (then St unused)
  uint8_t *mu;           // 32-byte slot per item
  uint32_t n, logq, B, pad;
};

struct MulSaArgs {
  const uint16_t *A;     // stored A (n x n) or NULL
  const uint8_t *seedA;  // fused: 16-byte seed (device)
  uint32_t n;
  uint32_t logq;
  const int8_t *S;       // item e: S (8 x n) at S + e * s_stride
  uint64_t s_stride;
  const int8_t *E;       // nullable, item e: 8 x n at E + e * e_stride
  uint64_t e_stride;
  uint8_t *out;          // item e rows at out + e*out_stride + 2 k n (uint16)
  uint64_t out_stride;
  uint32_t *flags;       // compare mode: atomicOr(flags[e], 1) on mismatch
  const uint16_t *const *A_ptrs;  // per-item stored A (then A unused)
  const uint8_t *const *seed_ptrs;  // per-item seedA at seed_ptrs[e] + seed_off (fused)
  uint64_t seed_off;
  // row block: the sum runs over rows [row0, row1) of A only (row1 = 0: n);
  // a stored A then points at row row0 (rows of length n)
  uint32_t row0, row1;
};

struct VEncArgs {
  const uint8_t *pk;     // seedA || B (n x 8 uint16)
  const uint8_t *const *pk_ptrs;  // per-item public key at pk_ptrs[e] + pk_off
  uint64_t pk_off;
  const int8_t *S;       // item e: S' (8 x n) at S + e * s_stride
  uint64_t s_stride;
  const int8_t *Epp;     // item e: E'' (8 x 8) at Epp + e * epp_stride
  uint64_t epp_stride;
  const uint8_t *mu;     // 32-byte slot per item
  uint8_t *ct;           // item e at ct + e * ct_bytes; C at +16n
  uint64_t ct_bytes;
  uint32_t *flags;
  uint32_t n, logq, B, pad;
};

struct KeygenSeedArgs {
  const uint8_t *ms;     // count x 32
  uint8_t *pk;
  uint8_t *sk;
  uint8_t *ws_seeds;     // count x 32: seedA || seedSE
  uint32_t *ws_rk;       // count x 44: round keys of seedSE
  uint64_t pk_bytes, sk_bytes;
  uint64_t sk_z_off, sk_pk_off;
  uint32_t count, pad;
};

struct DeriveArgs {
  const uint8_t *coins;  // Encaps: count x 32; Decaps: NULL (mu given)
  const uint8_t *pkh;    // 32 bytes
  const uint8_t *const *pkh_ptrs;  // per-item H(pk) at pkh_ptrs[e] + pkh_off
  uint64_t pkh_off;
  uint64_t pkh_stride;   // without pointers: H(pk) of item e at pkh + e * pkh_stride
  uint8_t *mu;           // 32-byte slot per item
  uint8_t *kprime;       // 32 per item
  uint8_t *seeds;        // 32-byte slot per item, seedSE' in the first 16
  uint32_t *rk;          // 44 round-key words of seedSE' per item
  uint32_t count, mu_bytes;
};

enum { TREE_DIGEST = 0, TREE_ENC_KEY = 1 };
#define TREE_MAX_THREADS 448  // 14 warps
#define TREE_WARP_MAX_THREADS 512  // 16 warps, one chunk each

// Tree hash of `count` messages of `len` bytes (item e at msgs + e*stride,
// or msg_ptrs[e]): leaves and root in one kernel, the leaf digests kept in
// shared memory.  DIGEST writes H to out + e*out_stride (and out2);
// ENC_KEY writes K = H(K'_e || H) to out + 32 e.
struct TreeArgs {
  const uint8_t *msgs;
  const uint8_t *const *msg_ptrs;
  uint64_t stride;
  uint32_t len, count;
  uint32_t m;            // leaves per message
  uint32_t tpi;          // threads per message (power of two <= 256)
  uint32_t ipc;          // messages per CTA
  uint32_t ml;           // full-length (1024-byte) chunks per message (k_tree_bal, k_tree_dense)
  uint32_t rw;           // k_tree_dense: the warp of the short chunks and roots
  int mode;
  uint8_t *out;
  uint64_t out_stride;
  uint8_t *out2;
  uint64_t out2_stride;
  const uint8_t *kprime; // 32 per item
  uint64_t *dig;         // scratch for the leaf digests of long messages
  uint64_t dig_words;    // (count x m x 4 words), or NULL / 0
};

// Decaps' key selection (Alg. 5): K = H(K' || H(c)) when the re-encryption
// matched (flag 0), else H(z || H(c)); branch-free.
struct FinalKeyArgs {
  const uint8_t *kprime; // 32 per item
  const uint8_t *hc;     // 32 per item
  const uint8_t *z;      // one key's z, or
  const uint8_t *const *z_ptrs;  // per item at z_ptrs[e] + z_off
  uint64_t z_off;
  const uint32_t *flags;
  uint8_t *K;
  uint32_t count, pad;
};

cudaError_t lwe_upload_aes_table(const uint32_t T0[256]);
cudaError_t lwe_kernel_smem_setup();
void launch_expand_A(const uint8_t *seeds, uint32_t seed_stride, uint32_t count, uint32_t n,
                     uint32_t logq, uint16_t *A, uint64_t a_stride, int num_sms, cudaStream_t st);
void launch_noise(const NoiseArgs &a, int num_sms, cudaStream_t st);
void launch_noise_table(const NoiseArgs &a, int8_t *out, cudaStream_t st);
void launch_mul_as(const MulAsArgs &a, uint32_t count, bool fused, int num_sms, cudaStream_t st);
void launch_decrypt(const DecryptArgs &a, uint32_t count, cudaStream_t st);
void launch_mul_sa(const MulSaArgs &a, uint32_t items, bool fused, bool cmp, int num_sms,
                   cudaStream_t st);
void launch_v_encode(const VEncArgs &a, uint32_t count, bool cmp, cudaStream_t st);
// launches of at most warp_max items hash with one Keccak state per warp
void launch_keygen_seeds(const KeygenSeedArgs &a, uint32_t warp_max, cudaStream_t st);
void launch_derive(const DeriveArgs &a, uint32_t warp_max, cudaStream_t st);
void launch_tree(TreeArgs &a, int num_sms, uint32_t warp_max, cudaStream_t st);
// bounds-checked build: skipped accesses of this unit's kernels (read and clear)
cudaError_t lwe_bounds_read_kem(unsigned long long *count, unsigned *site);
// measurement probes: kind 0 Keccak-f in registers (256-thread CTAs),
// kind 1 AES counter blocks with the shared-memory tables (512 threads)
int launch_probe(int kind, uint32_t ctas, uint32_t iters, uint32_t *sink, cudaStream_t st);
void launch_final_key(const FinalKeyArgs &a, uint32_t warp_max, cudaStream_t st);
