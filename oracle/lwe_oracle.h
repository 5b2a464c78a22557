/*
 * lwe_oracle.h -- plain CPU oracle of the plain-LWE KEM.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product links, loads or calls
 * this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg (and its `--impl reference` arm) may use it.  It shares no
 * source, header, table or helper with the CUDA library under
 * paper_2606_01211_gb300/csrc, and neither side includes the other.
 *
 * What it computes (citations are to the paper, arxiv 2606.01211):
 *   - KeyGen / Encrypt / Decrypt of Alg. 1-3 (Sec. 2.1) in matrix form:
 *       B  = A S + E              (Alg. 1, the LWE sample of Eq. 1)
 *       B' = S' A + E'            (Alg. 2, u = A^T r + e1 with r stacked)
 *       V  = S' B + E'',  C = V + Enc(mu)        (Alg. 2, v)
 *       M  = C - B' S,  mu' = Dec(M)             (Alg. 3)
 *   - Encaps / Decaps of Alg. 4-5 with the Fujisaki-Okamoto transform and
 *     implicit rejection (Sec. 2.1).
 *   - The seed expansion of A and of the noise on AES counter streams
 *     (Sec. 3.3), with AES-128 as defined in FIPS-197.
 *   - The hash H (unnamed in the paper) as SHA3-256 (FIPS 202), and, for the
 *     long inputs H(pk) and H(c), a fixed-shape two-level SHA3-256 tree.
 *
 * The paper leaves the concrete parameters, hash, counter format, sampler
 * table and byte layouts open; each reading taken here is listed in the
 * repository's design notes and stated beside the code that implements it.
 *
 * Parity status of each function:
 *   pinned   : AES-128 (FIPS-197 worked examples, independent AES library),
 *              SHA3-256 (independent hashlib), tree hash (composition of
 *              hashlib calls), CDF table (Gaussian mass from an independent
 *              normal CDF; exhaustive 2^16 sampler enumeration), products
 *              (brute force in numpy int64 + closed-form special cases),
 *              KEM invariants (Decaps(Encaps) = K, implicit rejection key,
 *              |B - A S| <= c, decryption-noise variance).
 *   parity unpinned: the seed-derivation domain bytes, the counter-block
 *              format and the byte layouts of pk/sk/ct are this project's
 *              own readings; they are fixed only by the oracle itself and by
 *              agreement with the independently written CUDA path.
 */
#ifndef LWE_ORACLE_H
#define LWE_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint32_t n;     /* LWE dimension, multiple of 8                          */
  uint32_t nbar;  /* columns of S (8)                                      */
  uint32_t mbar;  /* rows of S' (8)                                        */
  uint32_t logq;  /* D, q = 2^D, 2..16                                     */
  uint32_t B;     /* message bits per coefficient of C, 1..4, B < D       */
  uint32_t clip;  /* c: noise magnitude bound |e| <= c, 1..15              */
  double sigma;   /* standard deviation of the rounded Gaussian            */
} orc_params;

/* ---- primitives -------------------------------------------------------- */
void orc_aes128_key_expand(const uint8_t key[16], uint8_t rk[176]);
void orc_aes128_encrypt(const uint8_t rk[176], const uint8_t in[16],
                        uint8_t out[16]);
/* keystream block for (domain, index): AES_key(BE64(domain) || BE64(index)) */
void orc_ctr_block(const uint8_t rk[176], uint64_t domain, uint64_t index,
                   uint8_t out[16]);
/* Blocks first .. first + count - 1 of the stream (key, domain). */
void orc_ctr_stream(const uint8_t key[16], uint64_t domain, uint64_t first, size_t count,
                    uint8_t *out);
void orc_sha3_256(const uint8_t *msg, size_t len, uint8_t out[32]);
/* two-level tree: SHA3-256( SHA3-256(chunk_0) || ... || SHA3-256(chunk_m-1) ),
 * chunks of ORC_TREE_CHUNK bytes, the last one possibly shorter */
#define ORC_TREE_CHUNK 1024
void orc_htree(const uint8_t *msg, size_t len, uint8_t out[32]);

/* ---- sampler ----------------------------------------------------------- */
/* T[0..clip-1]; returns 0, or -1 if the table is not strictly increasing */
int orc_cdf_table(double sigma, uint32_t clip, uint16_t *T);
int orc_sample(uint16_t w, const uint16_t *T, uint32_t clip);
/* count samples of stream (key, domain): sample k uses word k%8 of block k/8 */
void orc_noise(const uint8_t key[16], uint64_t domain, const uint16_t *T,
               uint32_t clip, size_t count, int8_t *out);

/* ---- matrices ---------------------------------------------------------- */
/* A (n x n, row-major): A[i][j..j+7] = LE words of block i*n/8 + j/8, & (q-1) */
void orc_expand_A(const uint8_t seedA[16], uint32_t n, uint32_t logq,
                  uint16_t *A);
/* out (n x k) = A (n x n) * S + E, with S given transposed as St (k x n),
 * E (n x k, nullable).  mod 2^logq. */
void orc_mul_AS(uint32_t n, uint32_t k, uint32_t logq, const uint16_t *A,
                const int8_t *St, const int8_t *E, uint16_t *out);
/* out (m x ncol) = S (m x n) * X (n x ncol) + E (m x ncol, nullable) */
void orc_mul_SA(uint32_t m, uint32_t n, uint32_t ncol, uint32_t logq,
                const int8_t *S, const uint16_t *X, const int8_t *E,
                uint16_t *out);

/* ---- KEM --------------------------------------------------------------- */
size_t orc_pk_bytes(const orc_params *p);
size_t orc_sk_bytes(const orc_params *p);
size_t orc_ct_bytes(const orc_params *p);
size_t orc_mu_bytes(const orc_params *p);
/* returns 0, or -1 on invalid parameters */
int orc_check_params(const orc_params *p);
int orc_keygen(const orc_params *p, const uint8_t ms[32], uint8_t *pk,
               uint8_t *sk, uint16_t *A_out /* nullable, n x n */);
/* A: nullable; when given it must be expand_A(seedA of pk) (pk = (A, t) in
 * Alg. 1); when NULL it is regenerated from the seed inside pk. */
int orc_encaps(const orc_params *p, const uint8_t *pk, const uint16_t *A,
               const uint8_t coins[32], uint8_t *ct, uint8_t K[32]);
int orc_decaps(const orc_params *p, const uint8_t *sk, const uint16_t *A,
               const uint8_t *ct, uint8_t K[32]);

/* intermediates, for element-wise comparison with other implementations */
typedef struct {
  uint8_t mu[32];
  uint8_t pkh[32];
  uint8_t kprime[32];
  uint8_t seed_se[16];
  uint8_t hc[32];
  int8_t *Sp;    /* nullable, mbar x n  */
  int8_t *Ep;    /* nullable, mbar x n  */
  int8_t *Epp;   /* nullable, mbar x nbar */
  uint16_t *M;   /* decaps only, nullable, mbar x nbar */
  int eq;        /* decaps only: 1 when the re-encryption matched */
} orc_trace;
int orc_encaps_trace(const orc_params *p, const uint8_t *pk, const uint16_t *A,
                     const uint8_t coins[32], uint8_t *ct, uint8_t K[32],
                     orc_trace *tr);
int orc_decaps_trace(const orc_params *p, const uint8_t *sk, const uint16_t *A,
                     const uint8_t *ct, uint8_t K[32], orc_trace *tr);

/* batches over independent items; nthreads <= 0 means one thread */
int orc_keygen_batch(const orc_params *p, const uint8_t *ms, size_t count,
                     uint8_t *pk, uint8_t *sk, int nthreads);
int orc_encaps_batch(const orc_params *p, const uint8_t *pk, const uint16_t *A,
                     const uint8_t *coins, size_t count, uint8_t *ct,
                     uint8_t *K, int nthreads);
int orc_decaps_batch(const orc_params *p, const uint8_t *sk, const uint16_t *A,
                     const uint8_t *ct, size_t count, uint8_t *K,
                     int nthreads);
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
