/* lwe_pp.h -- the paper's own parameter profile (Tab. 1) of the plain-LWE
 * KEM: the scheme of Alg. 1-5 with a vector secret s in Z_q^n, an odd
 * modulus q in {3329, 12289, 65537}, and a 256-bit message m encrypted one
 * bit at a time (Alg. 2 for each bit: u_k = A^T r_k + e1_k, v_k = t^T r_k
 * + e2_k + m_k floor(q/2)), so one Encaps computes the 256 x n by n x n
 * product R^T A.  Distributions as in Tab. 1: s binomial (eta = 3); e, r,
 * e1 the rounded Gaussian of the CDF table (sigma, clipped at |e| <= clip);
 * e2 centred uniform on [-k, k].  Decoding (Alg. 3): bit k is 1 iff
 * q < 4 mu_k < 3q.
 *
 * Conventions as in lwe.h: device pointers owned by the caller, 16-byte
 * aligned; asynchronous on `stream`; status codes LWE_* (lwe.h).  A context
 * owns the per-call workspace (the 256 x n noise of Encrypt, hashes, round
 * keys) and serves one call at a time.
 *
 * Byte layouts (little-endian; entries mod q are uint32):
 *   pk = seedA[16] || t (n uint32)                         16 + 4n bytes
 *   sk = s (n int8) || z[32] || H(pk)[32] || pk             n + 80 + 4n
 *   ct = U^T (256 x n uint32, row k = u_k) || v (256 uint32) 1024 n + 1024
 * A (n x n uint32, row-major) is expanded from seedA by lwe_pp_expand_A or
 * returned by lwe_pp_keygen; Encaps and Decaps take it as an input.
 *
 * Readings where the paper is silent: A is uniform mod q by rejection
 * sampling of 32-bit AES-CTR words (stream domains 16..23); the noise
 * streams and seeds follow the matrix-form KEM of lwe.h (seedSE' = H(0x01
 * || H(pk) || m) derandomises Encrypt); H(c) = Htree(Htree(u_0) || ... ||
 * Htree(u_255) || Htree(v)) with Htree the 1024-byte-chunk tree hash of
 * lwe.h, so the multi-megabyte ciphertext hashes in parallel.
 */
#ifndef LWE_PP_H
#define LWE_PP_H

#include <stddef.h>
#include <stdint.h>

#include "lwe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint32_t n;      /* lattice dimension: a multiple of 64, 64 .. 65536     */
  uint32_t q;      /* odd modulus, 3 .. 65537                               */
  uint32_t k;      /* e2 is centred uniform on [-k, k], 1 .. 15             */
  uint32_t clip;   /* Gaussian samples satisfy |e| <= clip, 1 .. 15         */
  double sigma;    /* Gaussian width of e, r, e1                            */
} lwe_pp_params;

/* Tab. 1 rows: n = 512 (q 3329), 1024, 2048, 4096 (q 12289), 8192, 16384,
 * 32768 (q 65537), with the table's sigma and k and the largest clip whose
 * CDF table is valid. */
enum {
  LWE_PP512 = 0, LWE_PP1024 = 1, LWE_PP2048 = 2, LWE_PP4096 = 3,
  LWE_PP8192 = 4, LWE_PP16384 = 5, LWE_PP32768 = 6
};
int lwe_pp_params_preset(int id, lwe_pp_params *out);
/* LWE_OK when the parameters are supported (ranges above, a valid CDF
 * table); LWE_EINVAL otherwise. */
int lwe_pp_params_check(const lwe_pp_params *p);
size_t lwe_pp_pk_bytes(const lwe_pp_params *p);
size_t lwe_pp_sk_bytes(const lwe_pp_params *p);
size_t lwe_pp_ct_bytes(const lwe_pp_params *p);

typedef struct lwe_pp_ctx lwe_pp_ctx;
/* Allocates the workspace on `device`: about 2.6 KB per unit of n for the
 * noise, the bf16 copy of r and the K-split sums, plus 4 n^2 bytes for the
 * bf16 limbs of A; the only allocating call.  LWE_EINVAL, LWE_ENOMEM,
 * LWE_ECUDA. */
int lwe_pp_ctx_create(const lwe_pp_params *p, int device, lwe_pp_ctx **out);
int lwe_pp_ctx_destroy(lwe_pp_ctx *ctx);
/* Options.  LWE_PP_OPT_TENSOR: 1 (default) computes Encrypt's product
 * R^T A on the tensor cores (A split into two signed 8-bit limbs of its
 * centred value, exact bf16 tcgen05 GEMM in K passes, reduced mod q in the
 * epilogue); 0 on the CUDA cores (int32 multiply-adds).  LWE_PP_OPT_PDL: 1
 * launches the kernels of a call with programmatic stream serialisation (as
 * LWE_OPT_PDL of lwe.h); 0 (default): plain launches, measured faster for
 * these calls at n = 1024, 8192 and 32768. */
enum { LWE_PP_OPT_TENSOR = 0, LWE_PP_OPT_PDL = 1 };
int lwe_pp_ctx_set_option(lwe_pp_ctx *ctx, int option, int64_t value);

/* A = sample(seedA) (Alg. 1) into A (n x n uint32).  seedA: 16
 * device bytes. */
int lwe_pp_expand_A(const lwe_pp_params *p, const uint8_t *seedA, uint32_t *A, void *stream);

/* KeyGen (Alg. 1) from a 32-byte master seed (device): writes pk, sk and
 * A (required). */
int lwe_pp_keygen(lwe_pp_ctx *ctx, const uint8_t *seed32, uint8_t *pk, uint8_t *sk,
                  uint32_t *A, void *stream);
/* Encaps (Alg. 4) against pk with its A: m = H(0x4D || coins32), ct and the
 * 32-byte key K. */
int lwe_pp_encaps(lwe_pp_ctx *ctx, const uint8_t *pk, const uint32_t *A, const uint8_t *coins32,
                  uint8_t *ct, uint8_t *K, void *stream);
/* Per-key precomputation for repeated calls against one key: H(pk) (Alg.
 * 4 hashes pk in every Encaps) and, on the tensor path, the bf16 limb split
 * of A (4 n^2 bytes read and written per call otherwise: 8 GiB of memory
 * traffic at n = 32768).  Later lwe_pp_encaps calls with this pk pointer
 * skip H(pk), and lwe_pp_encaps / lwe_pp_decaps calls with this A pointer
 * skip the limb split; results are identical.  pk and A nullable (both NULL
 * unbinds).  The binding refers to the buffers: their contents must not
 * change while bound.  A call with another A overwrites the limbs and the
 * next call with the bound A makes them again.  Order later calls after
 * this call's work; allocates nothing.  LWE_EINVAL for a NULL context or
 * misaligned pointers. */
int lwe_pp_ctx_bind_key(lwe_pp_ctx *ctx, const uint8_t *pk, const uint32_t *A, void *stream);

/* Decaps (Alg. 5): K = H(K' || H(c)) when the re-encryption reproduces ct,
 * else H(z || H(c)) (implicit rejection, not an error). */
int lwe_pp_decaps(lwe_pp_ctx *ctx, const uint8_t *sk, const uint32_t *A, const uint8_t *ct,
                  uint8_t *K, void *stream);

#ifdef __cplusplus
}
#endif
#endif
