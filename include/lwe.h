/*
 * lwe.h -- C ABI of the GB300 (sm_103a) plain-LWE KEM library (liblwe.so).
 *
 * The scheme is the plain-LWE key encapsulation mechanism of arxiv
 * 2606.01211 (Liberati et al.), Sec. 2.1, Alg. 1-5, written in matrix form
 * with nbar = mbar = 8:
 *
 *   KeyGen   (Alg. 1):  A <- sample(seedA);  S, E <- chi;  B = A S + E mod q
 *   Encrypt  (Alg. 2):  S', E', E'' <- chi;  B' = S' A + E';  V = S' B + E'';
 *                       C = V + Enc(mu)
 *   Decrypt  (Alg. 3):  M = C - B' S;  mu = Dec(M)
 *   Encaps   (Alg. 4):  c = Encrypt(pk, mu);  K = H(H(H(pk) || mu) || H(c))
 *   Decaps   (Alg. 5):  re-encrypt and compare; on mismatch K = H(z || H(c))
 *                       (Fujisaki-Okamoto transform with implicit rejection)
 *
 * q = 2^logq.  A is expanded from a 16-byte seed with AES-128 in counter
 * mode on the device (Sec. 3.3: device-resident random number generation);
 * the noise is drawn from a rounded-Gaussian CDF table by inverse sampling
 * of the same kind of counter stream.
 *
 * Conventions shared by every entry point below:
 *   - Every buffer argument is a DEVICE pointer (cudaMalloc'd or a torch
 *     tensor's storage) owned by the caller, unless marked "host".  The
 *     library never frees or keeps caller buffers.
 *   - Buffers must be 16-byte aligned.  Misaligned or NULL required
 *     pointers return LWE_EINVAL before anything is launched.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is asynchronous on that stream: results are
 *     valid once the stream has been synchronised.  The calls enqueue work
 *     and return; they never synchronise the device and never allocate
 *     device memory (workspaces belong to the lwe_ctx and are sized when it
 *     is created).
 *   - Return value: LWE_OK (0) or a negative LWE_E* code.  Launch failures
 *     surface as LWE_ECUDA (the CUDA error string is kept for
 *     lwe_last_cuda_error()).  Waits inside kernels are bounded; a wait that
 *     runs out sets the context's device error word (LWE_ETIMEOUT), read by
 *     lwe_ctx_device_error().
 *   - Byte layouts (all integers little-endian):
 *       pk = seedA[16] || B (n x 8 uint16, row-major)
 *       sk = S^T (8 x n int8, row-major) || z[32] || H(pk)[32] || pk
 *       ct = B' (8 x n uint16, row-major) || C (8 x 8 uint16, row-major)
 *       K  = 32 bytes
 *     Batches are these objects back to back (item i at i * size).
 *   - The library requires n % 16 == 0 and 16 <= n <= 65536.
 */
#ifndef LWE_H
#define LWE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LWE_OK 0
#define LWE_EINVAL (-1)       /* bad argument, size, pointer or alignment */
#define LWE_ENOMEM (-2)       /* workspace allocation failed (create only)  */
#define LWE_ECUDA (-3)        /* a CUDA runtime call or launch failed       */
#define LWE_ETIMEOUT (-4)     /* a bounded device wait ran out              */
#define LWE_EUNSUPPORTED (-5) /* not supported on this device               */
#define LWE_ECAPACITY (-6)    /* count exceeds the context's max_batch, or
                                 (lwe_encaps_noalloc) the built-in scratch  */

/* ---- parameters (Sec. 2.2; the values of the presets are the workloads'
 *      parameter sets, each with nbar = mbar = 8) -------------------------- */
typedef struct lwe_params {
  uint32_t n;     /* LWE dimension                                         */
  uint32_t nbar;  /* columns of S, must be 8                               */
  uint32_t mbar;  /* rows of S', must be 8                                 */
  uint32_t logq;  /* q = 2^logq, 2..16                                     */
  uint32_t B;     /* message bits per coefficient of C, 1..4, B < logq    */
  uint32_t clip;  /* noise bound c: samples lie in [-c, c], 1..15          */
  double sigma;   /* standard deviation of the rounded Gaussian           */
} lwe_params;

enum {
  LWE_P640 = 0,   /* n=640,   q=2^15, sigma=2.8, c=12, B=2 */
  LWE_P976 = 1,   /* n=976,   q=2^16, sigma=2.3, c=10, B=3 */
  LWE_P1344 = 2,  /* n=1344,  q=2^16, sigma=1.4, c=6,  B=4 */
  LWE_P4096 = 3,  /* n=4096,  q=2^16, sigma=2.8, c=12, B=2 */
  LWE_P16384 = 4, /* n=16384, q=2^16, sigma=2.8, c=12, B=1 */
  LWE_P32768 = 5  /* n=32768, q=2^16, sigma=2.8, c=12, B=1 */
};

/* Fill *out with preset `id`.  Host only.  LWE_EINVAL for an unknown id. */
int lwe_params_preset(int id, lwe_params *out);

/* LWE_OK when *p is usable by this library (see the ranges above and the
 * table condition of lwe_cdf_table).  Host only. */
int lwe_params_check(const lwe_params *p);

/* The inverse-sampling table of the noise distribution (Sec. 2.2, Tab. 1:
 * Gaussian noise of width sigma).  Reading of the paper: p(k) is the mass
 * of N(0, sigma^2) on [k - 1/2, k + 1/2] for |k| <= c, renormalised;
 * T[k] = round_half_up(2^15 * (p(0) + 2 sum_{j=1..k} p(j))) - 1, k < c.
 * A sample takes a 16-bit word w: t = w >> 1, |e| = #{k : t > T[k]},
 * e < 0 iff w & 1.  Host only; writes T[0..clip-1].  LWE_EINVAL if the
 * table is not strictly increasing or its last entry reaches 2^15 - 1. */
int lwe_cdf_table(const lwe_params *p, uint16_t T[16]);

/* Object sizes in bytes. Host only. */
size_t lwe_pk_bytes(const lwe_params *p);
size_t lwe_sk_bytes(const lwe_params *p);
size_t lwe_ct_bytes(const lwe_params *p);

/* ---- context ----------------------------------------------------------- */
typedef struct lwe_ctx lwe_ctx;

/* Create a context for parameters *p on CUDA device `device`, with
 * workspaces for up to `max_batch` items per call (>= 1).  This is the only
 * call that allocates device memory; it also uploads the AES table to the
 * device and must not run during stream capture.  *out is set to NULL on
 * failure.  Returns LWE_EINVAL, LWE_ENOMEM, LWE_ECUDA or LWE_EUNSUPPORTED
 * (device is not sm_103). */
int lwe_ctx_create(const lwe_params *p, uint32_t max_batch, int device,
                   lwe_ctx **out);
/* Free the context and its workspaces (synchronises the device first).
 * NULL is accepted. */
int lwe_ctx_destroy(lwe_ctx *ctx);

/* Product path for Encrypt's S' A (Alg. 2): */
enum {
  LWE_PATH_AUTO = 0,   /* tensor path when count >= the tuned threshold  */
  LWE_PATH_SKINNY = 1, /* per-item CUDA-core kernels ("plain" path)      */
  LWE_PATH_TENSOR = 2  /* stacked S' as one exact two-limb bf16 tcgen05
                          GEMM (tensor cores, fp32 accumulation; K split
                          into passes of at most (2^24-1)/(128 c) columns).
                          Available for n <= 8192, or for larger n when the
                          context was created with max_batch >= 64.       */
};
enum {
  LWE_OPT_PATH = 0,          /* one of LWE_PATH_*                             */
  LWE_OPT_TENSOR_MIN = 1,    /* AUTO threshold (items per call), default 64   */
  LWE_OPT_TIMING = 2,        /* 1: time every launch with CUDA events          */
  LWE_OPT_GEMM_BN = 3,       /* single-CTA GEMM column tile: 64 or 128 (def.) */
  LWE_OPT_GEMM_KCHUNK = 4,   /* K per tensor-core pass: a multiple of 64 up to
                                the exact bound (2^24-1)/(128 c); 0 = bound   */
  LWE_OPT_GEMM_PAIR = 5,     /* 1 (default): the GEMM runs on CTA pairs (two
                                SMs share a 256 x 128 tile, tcgen05
                                cta_group::2; LWE_OPT_GEMM_BN is then
                                ignored); 0: one CTA per 128 x BN tile        */
  LWE_OPT_SERIAL = 6,        /* 1: work that normally overlaps on the
                                context's side stream (the tensor path's
                                limbs, Decaps' H(c)) runs on the caller's
                                stream, so that per-kernel timings measure
                                each kernel alone; 0 (default): overlapped   */
  LWE_OPT_WARP_HASH_MAX = 7, /* hashing launches (tree hashes H(pk), H(c);
                                KeyGen seeds; mu, K', seedSE'; the Decaps
                                key) of at most this many items run with
                                one Keccak state per warp (the lanes of
                                the state spread over the threads: lower
                                latency), larger ones with one state per
                                thread (higher throughput).  -1 (default):
                                the number of SMs; 0: always per thread   */
  LWE_OPT_PDL = 8,           /* 1 (default): the kernels of Encaps / Decaps
                                are launched with programmatic stream
                                serialisation (each may start while the
                                previous one drains, and waits on the
                                device for its results); 0: plain launches */
  LWE_OPT_GEMM_GROUP = 9     /* tensor-core GEMM tile order: the persistent
                                CTAs visit output tiles in groups of this
                                many row blocks of S' (the row block varies
                                fastest inside a group), 1..64; 1 is plain
                                row-major order.  0 (default): 1 while one
                                pass's [A | B] limbs fit in 32 MB (they stay
                                in L2), else 8 (each limb tile is then read
                                from HBM once per 8 row blocks instead of
                                once per row block).  Results never depend
                                on it. */
};
int lwe_ctx_set_option(lwe_ctx *ctx, int option, int64_t value);

/* ---- KEM (Alg. 1, 4, 5) ------------------------------------------------ */

/* KeyGen, Alg. 1, for `count` independent key pairs.
 *   seeds  [count][32]         master seeds.  Derived: seedA =
 *                              H(0x41||ms)[0:16], seedSE = H(0x53||ms)[0:16],
 *                              z = H(0x5A||ms) with H = SHA3-256.
 *   pk     [count][pk_bytes]   output.
 *   sk     [count][sk_bytes]   output.
 *   A_out  [count][n][n] uint16, nullable: when given, A is written there
 *          (stored mode); when NULL it is regenerated inside the product and
 *          never stored (Sec. 3.5, Sec. 4.3: on-demand generation of A).
 * count == 0 is a no-op.  count > max_batch returns LWE_ECAPACITY. */
int lwe_keygen(lwe_ctx *ctx, const uint8_t *seeds, uint32_t count,
               uint8_t *pk, uint8_t *sk, uint16_t *A_out, void *stream);

/* Encaps, Alg. 4 (with Encrypt of Alg. 2), `count` encapsulations against
 * ONE public key.
 *   pk     [pk_bytes]           public key.
 *   A      [n][n] uint16, nullable: the expansion of pk's seedA (stored
 *          mode); NULL regenerates A on the fly.
 *   coins  [count][32]          randomness: mu = H(0x4D||coins)[0:8B bytes].
 *   ct     [count][ct_bytes]    output ciphertexts.
 *   K      [count][32]          output shared keys. */
int lwe_encaps(lwe_ctx *ctx, const uint8_t *pk, const uint16_t *A,
               const uint8_t *coins, uint32_t count, uint8_t *ct, uint8_t *K,
               void *stream);

/* Decaps, Alg. 5 (with Decrypt of Alg. 3), `count` decapsulations with ONE
 * secret key.  Constant time in the validity of each ciphertext: the
 * re-encryption is compared with a branch-free OR of differences and the
 * key material is selected by masking (implicit rejection, Sec. 2.1).
 *   sk  [sk_bytes];  A as in lwe_encaps (pk is taken from inside sk);
 *   ct  [count][ct_bytes];  K [count][32] output. */
int lwe_decaps(lwe_ctx *ctx, const uint8_t *sk, const uint16_t *A,
               const uint8_t *ct, uint32_t count, uint8_t *K, void *stream);

/* Encaps / Decaps of `count` items that each use their OWN key (a server
 * batching requests across keys).  Item e uses:
 *   pk_ptrs[e]  (Encaps)  device array of count device pointers to pk;
 *   pkh_ptrs[e] (Encaps)  nullable device array of pointers to H(pk)
 *               (32 bytes, e.g. inside the matching sk); NULL computes it;
 *   sk_ptrs[e]  (Decaps)  device array of count device pointers to sk;
 *   A_ptrs[e]   nullable device array of pointers to each item's stored A;
 *               NULL regenerates every item's A from its seed.  A batch is
 *               either all-stored or all-regenerated.
 * coins / ct / K are laid out as in lwe_encaps / lwe_decaps.  Results are
 * identical to one single-key call per item.  These calls always take the
 * CUDA-core product (the tensor path needs one shared A).  Pointer arrays
 * must be 8-byte aligned, key objects 16-byte aligned. */
int lwe_encaps_multi(lwe_ctx *ctx, const uint8_t *const *pk_ptrs,
                     const uint8_t *const *pkh_ptrs, const uint16_t *const *A_ptrs,
                     const uint8_t *coins, uint32_t count, uint8_t *ct,
                     uint8_t *K, void *stream);
int lwe_decaps_multi(lwe_ctx *ctx, const uint8_t *const *sk_ptrs,
                     const uint16_t *const *A_ptrs, const uint8_t *ct,
                     uint32_t count, uint8_t *K, void *stream);

/* Per-key precomputation for repeated calls against one key pair.  Encaps
 * (Alg. 4) needs H(pk) for every call, and the tensor path multiplies by the
 * limb split of [A | B]; both depend on the key only.  Binding a key makes
 * them once, on `stream`; later lwe_encaps calls whose (pk, A) pointers
 * equal the bound (pk, A), and lwe_decaps calls whose (sk, A) equal the
 * bound (sk, A), reuse them instead of recomputing.  Results are identical
 * with and without a binding.
 *   pk  [pk_bytes] nullable;  sk [sk_bytes] nullable (at least one given;
 *       when both are given they must be the two halves of one key pair);
 *   A   [n][n] uint16 nullable, as in lwe_encaps.
 * pk = sk = NULL unbinds.  The binding refers to the BUFFERS: while a key is
 * bound their contents must not change (bind again after rewriting them).
 * Other calls on the context that need the limb workspace (a tensor-path
 * call for another key, lwe_matmul_modq) overwrite it; the next bound call
 * then makes the limbs again, on its own.  A CUDA graph captured from
 * bound calls reads the limbs the binding left in the workspace: do not let
 * another call overwrite them while such a graph is replayed.  Order later
 * calls after this call's work (same stream, or synchronise).  Allocates
 * nothing.
 * LWE_EINVAL for a NULL context or a misaligned pointer. */
int lwe_ctx_bind_key(lwe_ctx *ctx, const uint8_t *pk, const uint8_t *sk,
                     const uint16_t *A, void *stream);

/* ---- standalone hot-path kernels --------------------------------------- */

/* sample(seedA) of Alg. 1: A[i][j..j+7] = the eight little-endian 16-bit
 * words of AES-128_{seedA}(BE64(0) || BE64(i*n/8 + j/8)), each masked to
 * logq bits.  seedA [16] device; A_out [n][n] uint16 device.
 * Written with coalesced 16-byte stores.  Needs no context. */
int lwe_expand_A(const uint8_t *seedA, uint32_t n, uint32_t logq,
                 uint16_t *A_out, void *stream);

/* The mod-q products of Alg. 1-2 on their own (q = 2^logq):
 *   side LWE_SIDE_AS:  out[n][k]  = A S  + E,  S given as S^T [k][n] int8,
 *                      E [n][k] int8 (nullable); k must be 8.
 *   side LWE_SIDE_SA:  out[k][n]  = S A  + E,  S [k][n] int8,
 *                      E [k][n] int8 (nullable); k a multiple of 8
 *                      (k = 8 * stacked encryptions).
 * A [n][n] uint16, or NULL to regenerate it from seedA [16] (device) tile
 * by tile inside the product, never storing it.  ctx: nullable; when given
 * (and its n equals n and its max_batch covers k/8), SA may take the
 * tensor-core path and its workspace -- then every |S| must be at most the
 * context's clip, which bounds the exact K per tensor-core pass; otherwise
 * the CUDA-core kernels run. */
enum { LWE_SIDE_AS = 0, LWE_SIDE_SA = 1 };
int lwe_matmul_modq(lwe_ctx *ctx, int side, const uint16_t *A,
                    const uint8_t *seedA, const int8_t *S, uint32_t n,
                    uint32_t k, uint32_t logq, const int8_t *E,
                    uint16_t *out, void *stream);

/* The same products restricted to a block of rows of A, for one huge-n
 * operation split over several GPUs (the paper names multi-GPU execution
 * as future work, Sec. 5; Sec. 4.3 shows the large-n products are bound by
 * A's memory traffic or its regeneration).  Each GPU holds or regenerates
 * only rows [row0, row1) of A:
 *   side LWE_SIDE_AS:  out[row1 - row0][8] = rows row0 .. row1-1 of A S + E,
 *                      E given for those rows only ([row1 - row0][8],
 *                      nullable); the blocks of all GPUs, gathered in row
 *                      order, are B = A S + E.
 *   side LWE_SIDE_SA:  out[k][n] = (S[:, row0:row1] A[row0:row1, :] + E)
 *                      mod q, a partial sum over the block's rows (E
 *                      nullable, k x n: give it on one GPU only); summing
 *                      the partials of all GPUs (as integers) and reducing
 *                      mod q gives S A + E.
 * A_rows [row1 - row0][n] uint16: the block of rows (row row0 first), or
 * NULL to regenerate those rows from seedA [16] (device).  S as in
 * lwe_matmul_modq (S^T [8][n] for AS, S [k][n] for SA, full width).  row0
 * and row1 multiples of 16 with row0 < row1 <= n.  CUDA-core kernels;
 * needs no context.  LWE_EINVAL for bad sizes or pointers. */
int lwe_matmul_modq_rows(int side, const uint16_t *A_rows, const uint8_t *seedA,
                         const int8_t *S, uint32_t n, uint32_t k, uint32_t logq,
                         uint32_t row0, uint32_t row1, const int8_t *E, uint16_t *out,
                         void *stream);

/* ---- Encaps without any device allocation ------------------------------ */

/* Size of the library's built-in scratch area.  Every GPU that loads
 * liblwe.so keeps this much device memory reserved until the process exits. */
#define LWE_NOALLOC_SCRATCH_BYTES (1024u * 1024u)

/* Encaps exactly as lwe_encaps (same inputs, outputs, layouts and results;
 * CUDA-core path), for callers that cannot allocate device memory and so
 * cannot create an lwe_ctx: code that must not call cudaMalloc/cudaFree
 * because the host application owns every device allocation through its own
 * pool, or because a request path cannot afford an allocation's implicit
 * synchronisation and latency.  The paper has no counterpart; this is a
 * deployment convenience.
 *
 * Instead of a context workspace it uses one fixed scratch area compiled
 * into the library (LWE_NOALLOC_SCRATCH_BYTES on each device).  The caller
 * still passes every input and output buffer; the call makes no cudaMalloc,
 * cudaFree or other allocating call.  It runs on the CURRENT device; the
 * first call on a device looks up the scratch area's device address and
 * uploads the AES table there (one-time set-up), so make that first call
 * outside any stream capture.  The scratch holds about
 *   count * (16 n + 352) bytes
 * (each part rounded up to 256 bytes); a (params, count) that does not fit
 * returns LWE_ECAPACITY, invalid parameters or pointers LWE_EINVAL.
 * All calls on a device share the one area and it keeps the last call's
 * contents: every byte a call reads is written by that same call first, but
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads) race on it and give wrong results — serialise them. */
int lwe_encaps_noalloc(const lwe_params *p, const uint8_t *pk,
                       const uint16_t *A, const uint8_t *coins, uint32_t count,
                       uint8_t *ct, uint8_t *K, void *stream);

/* ---- diagnostics ------------------------------------------------------- */
const char *lwe_strerror(int code);
/* The last CUDA error string seen by this thread's calls ("" if none). */
const char *lwe_last_cuda_error(void);
/* Synchronises the device, returns LWE_OK or the device error word set by
 * a bounded wait (LWE_ETIMEOUT), and clears it. */
int lwe_ctx_device_error(lwe_ctx *ctx);
/* Number of kernels this context has launched so far. */
uint64_t lwe_ctx_launches(const lwe_ctx *ctx);
/* Failure-detection self-test (no counterpart in the paper): launches one
 * tiny kernel that waits, through the same bounded mbarrier wait the tensor
 * path uses, on a barrier that nothing ever completes.  The wait gives up
 * after limit_us microseconds (1 .. 2,000,000), raises the context's device
 * error word and the kernel returns normally -- nothing faults or hangs, and
 * the next lwe_ctx_device_error() returns LWE_ETIMEOUT (and clears it). */
int lwe_selftest_bounded_wait(lwe_ctx *ctx, uint32_t limit_us, void *stream);

/* The noise sampler's word table exactly as the noise kernel builds and
 * reads it (Sec. 2.2, Tab. 1: the rounded-Gaussian inverse sampling of
 * lwe_cdf_table): out[w] = e for every 16-bit word w, 65536 int8 values
 * (device).  A check of the device-side table against the sampler's
 * definition; one CTA, asynchronous on `stream`.  LWE_EINVAL for invalid
 * parameters or a NULL out. */
int lwe_noise_table(const lwe_params *p, int8_t *out, void *stream);

/* Bounds-checked debug build (no counterpart in the paper; a stand-in for
 * a memory checker): liblwe_check.so, the same library compiled with
 * LWE_CHECK_BOUNDS, makes every kernel test the index arithmetic of its
 * memory accesses against the sizes it was given and skip, instead of make,
 * an access that would leave its buffer.  This call synchronises the
 * device and returns in *count the number of accesses skipped since the
 * previous call (then clears it) and in *first_site an id of the first
 * failing site (0 if none).  The product build (liblwe.so) has no checks
 * and returns LWE_EUNSUPPORTED; LWE_EINVAL for NULL pointers. */
int lwe_bounds_violations(uint64_t *count, uint32_t *first_site);

/* Measurement probes (no counterpart in the paper): the instruction
 * sequences of the two integer-bound kernels without memory traffic, to
 * measure their practical peak on the current device.
 *   LWE_PROBE_KECCAK: `ctas` CTAs of 256 threads; each thread applies
 *     Keccak-f[1600] `iters` times to a state held in registers (the
 *     permutation of k_tree).  Work: ctas * 256 * iters permutations.
 *   LWE_PROBE_AES: `ctas` CTAs of 512 threads with the AES round tables in
 *     shared memory; each thread encrypts `iters` (even) counter blocks, two
 *     at a time, every round in full (the generator of the kernels whose
 *     blocks do not run along one counter window, e.g. S' A with A
 *     regenerated).  Work: ctas * 512 * iters blocks.
 *   LWE_PROBE_AES_RUN: as LWE_PROBE_AES with the blocks of a warp taken
 *     four per lane from one 128-block run of counter indices, whose first
 *     two rounds are shared, the constants of 32 runs worked out at once,
 *     under one key per warp (the generator of the noise and of A); iters
 *     a multiple of 4.
 *   LWE_PROBE_KECCAK_WARP: `ctas` CTAs of one warp; each warp applies
 *     Keccak-f[1600] `iters` times to one state spread over its lanes (the
 *     permutation of k_tree_warp).  Work: ctas * iters permutations.
 * One word per thread is written to sink (device, >= ctas * 512 words) so
 * that the work is kept.  Asynchronous on `stream`; time it with CUDA events
 * there.  LWE_EINVAL for an unknown kind, ctas = 0, or iters not a multiple
 * of 2 (AES) or 4 (AES_RUN). */
enum { LWE_PROBE_KECCAK = 0, LWE_PROBE_AES = 1, LWE_PROBE_KECCAK_WARP = 2, LWE_PROBE_AES_RUN = 3 };
int lwe_probe(int kind, uint32_t ctas, uint32_t iters, uint32_t *sink, void *stream);

/* Per-kernel event timing (needs LWE_OPT_TIMING = 1; synchronises). */
int lwe_ctx_kernel_stats(lwe_ctx *ctx, int kernel_id, uint64_t *launches,
                         double *total_ms);
int lwe_ctx_reset_stats(lwe_ctx *ctx);
/* Timing of launches captured into a CUDA graph: after capturing with
 * LWE_OPT_TIMING = 1, lwe_ctx_timing_mark keeps the captured event pairs
 * (their records are graph nodes, re-recorded by every replay); after each
 * replay has completed, lwe_ctx_timing_replay adds their durations to the
 * per-kernel statistics.  Marking again releases the previous pairs. */
int lwe_ctx_timing_mark(lwe_ctx *ctx);
int lwe_ctx_timing_replay(lwe_ctx *ctx);
/* Name of kernel id 0..lwe_num_kernels()-1, NULL out of range. */
const char *lwe_kernel_name(int kernel_id);
int lwe_num_kernels(void);

#ifdef __cplusplus
}
#endif
#endif /* LWE_H */
