/*
 * lwe_oracle.c -- plain, slow, obviously correct CPU oracle of the
 * plain-LWE KEM.  TEST INFRASTRUCTURE ONLY (see lwe_oracle.h): only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may use it.
 *
 * Everything here is scalar C written from the definitions: AES-128 from
 * FIPS-197 (S-box derived from the GF(2^8) inverse and the affine map, no
 * lookup tables of round functions), Keccak-f[1600] / SHA3-256 from FIPS 202
 * (rotation offsets and round constants derived from their defining
 * recurrences), the rounded-Gaussian CDF table from the normal CDF, and the
 * KEM from Alg. 1-5 of the paper in the matrix form B = A S + E.
 *
 * Parity unpinned: the domain bytes of the seed derivation, the domain
 * numbering of the counter blocks and the pk / sk / ct byte layouts are
 * readings of this project (the paper fixes none of them); nothing but this
 * oracle fixes them.  Every function built on them is pinned otherwise
 * (tests/test_oracle_pins.py).
 */
#include "lwe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ======================================================================== */
/* AES-128, FIPS-197                                                         */
/* ======================================================================== */

/* multiplication in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1 (FIPS-197 4.2) */
static uint8_t gf_mul(uint8_t a, uint8_t b) {
  uint8_t r = 0;
  for (int i = 0; i < 8; i++) {
    if (b & 1) r ^= a;
    uint8_t hi = a & 0x80;
    a = (uint8_t)(a << 1);
    if (hi) a ^= 0x1b;
    b >>= 1;
  }
  return r;
}

static uint8_t xtime(uint8_t a) { return gf_mul(a, 2); }

static uint8_t SBOX[256];
static int sbox_ready = 0;

/* S-box (FIPS-197 5.1.1): multiplicative inverse in GF(2^8) (0 -> 0)
 * followed by the affine transformation with constant 0x63. */
static void build_sbox(void) {
  for (int x = 0; x < 256; x++) {
    uint8_t inv = 0;
    if (x != 0) {
      for (int y = 1; y < 256; y++) {
        if (gf_mul((uint8_t)x, (uint8_t)y) == 1) {
          inv = (uint8_t)y;
          break;
        }
      }
    }
    uint8_t s = 0;
    for (int i = 0; i < 8; i++) {
      int bit = ((inv >> i) & 1) ^ ((inv >> ((i + 4) % 8)) & 1) ^
                ((inv >> ((i + 5) % 8)) & 1) ^ ((inv >> ((i + 6) % 8)) & 1) ^
                ((inv >> ((i + 7) % 8)) & 1) ^ ((0x63 >> i) & 1);
      s |= (uint8_t)(bit << i);
    }
    SBOX[x] = s;
  }
  sbox_ready = 1;
}

static uint8_t sub_byte(uint8_t x) {
  if (!sbox_ready) build_sbox();
  return SBOX[x];
}

/* KeyExpansion (FIPS-197 5.2): 44 words, Rcon[i] = x^(i-1) in GF(2^8). */
void orc_aes128_key_expand(const uint8_t key[16], uint8_t rk[176]) {
  if (!sbox_ready) build_sbox();
  memcpy(rk, key, 16);
  uint8_t rcon = 1;
  for (int i = 4; i < 44; i++) {
    uint8_t t[4];
    memcpy(t, rk + 4 * (i - 1), 4);
    if (i % 4 == 0) {
      uint8_t r0 = t[0];  /* RotWord */
      t[0] = t[1];
      t[1] = t[2];
      t[2] = t[3];
      t[3] = r0;
      for (int b = 0; b < 4; b++) t[b] = sub_byte(t[b]);  /* SubWord */
      t[0] ^= rcon;
      rcon = xtime(rcon);
    }
    for (int b = 0; b < 4; b++) rk[4 * i + b] = rk[4 * (i - 4) + b] ^ t[b];
  }
}

/* Cipher (FIPS-197 5.1): state s[r][c] = in[r + 4c]. */
void orc_aes128_encrypt(const uint8_t rk[176], const uint8_t in[16],
                        uint8_t out[16]) {
  uint8_t s[4][4];
  for (int c = 0; c < 4; c++)
    for (int r = 0; r < 4; r++) s[r][c] = in[r + 4 * c] ^ rk[r + 4 * c];
  for (int round = 1; round <= 10; round++) {
    /* SubBytes */
    for (int r = 0; r < 4; r++)
      for (int c = 0; c < 4; c++) s[r][c] = sub_byte(s[r][c]);
    /* ShiftRows: row r rotates left by r */
    for (int r = 1; r < 4; r++) {
      uint8_t t[4];
      for (int c = 0; c < 4; c++) t[c] = s[r][(c + r) % 4];
      for (int c = 0; c < 4; c++) s[r][c] = t[c];
    }
    /* MixColumns, skipped in the final round */
    if (round != 10) {
      for (int c = 0; c < 4; c++) {
        uint8_t a0 = s[0][c], a1 = s[1][c], a2 = s[2][c], a3 = s[3][c];
        s[0][c] = gf_mul(a0, 2) ^ gf_mul(a1, 3) ^ a2 ^ a3;
        s[1][c] = a0 ^ gf_mul(a1, 2) ^ gf_mul(a2, 3) ^ a3;
        s[2][c] = a0 ^ a1 ^ gf_mul(a2, 2) ^ gf_mul(a3, 3);
        s[3][c] = gf_mul(a0, 3) ^ a1 ^ a2 ^ gf_mul(a3, 2);
      }
    }
    /* AddRoundKey */
    for (int c = 0; c < 4; c++)
      for (int r = 0; r < 4; r++) s[r][c] ^= rk[16 * round + r + 4 * c];
  }
  for (int c = 0; c < 4; c++)
    for (int r = 0; r < 4; r++) out[r + 4 * c] = s[r][c];
}

/* Counter block for (domain, index): BE64(domain) || BE64(index). */
void orc_ctr_block(const uint8_t rk[176], uint64_t domain, uint64_t index,
                   uint8_t out[16]) {
  uint8_t in[16];
  for (int b = 0; b < 8; b++) {
    in[b] = (uint8_t)(domain >> (56 - 8 * b));
    in[8 + b] = (uint8_t)(index >> (56 - 8 * b));
  }
  orc_aes128_encrypt(rk, in, out);
}

/* `count` consecutive keystream blocks (domain, first .. first + count - 1)
 * under one key, for the paper-profile oracle's long streams. */
void orc_ctr_stream(const uint8_t key[16], uint64_t domain, uint64_t first, size_t count,
                    uint8_t *out) {
  uint8_t rk[176];
  orc_aes128_key_expand(key, rk);
  for (size_t b = 0; b < count; b++) orc_ctr_block(rk, domain, first + b, out + 16 * b);
}

/* ======================================================================== */
/* Keccak-f[1600] and SHA3-256, FIPS 202                                     */
/* ======================================================================== */

static uint64_t rotl64(uint64_t x, unsigned r) {
  r &= 63;
  return r ? (x << r) | (x >> (64 - r)) : x;
}

static int keccak_ready = 0;
static unsigned RHO[25];   /* rotation offset of lane x + 5y   */
static uint64_t RC[24];    /* round constants                   */

/* rc(t) of FIPS 202 Algorithm 5: the LFSR x^8 + x^6 + x^5 + x^4 + 1 */
static int rc_bit(int t) {
  if (t % 255 == 0) return 1;
  uint8_t R = 0x80;  /* R = 10000000, leftmost bit is R[0] */
  for (int i = 1; i <= t % 255; i++) {
    /* R = 0 || R, then R[0]^=R[8], R[4]^=R[8], R[5]^=R[8], R[6]^=R[8],
     * then truncate to 8 bits.  With R[0] as the most significant bit of
     * the byte, prepending 0 is a right shift and R[8] is the bit shifted
     * out. */
    int r8 = R & 1;
    R >>= 1;
    if (r8) R ^= 0x80 | 0x08 | 0x04 | 0x02;
  }
  return (R >> 7) & 1;
}

static void build_keccak(void) {
  /* rho offsets (FIPS 202 3.2.2): (x,y) = (1,0); for t = 0..23 the lane
   * (x,y) rotates by (t+1)(t+2)/2 mod 64, then (x,y) = (y, 2x+3y mod 5). */
  memset(RHO, 0, sizeof RHO);
  int x = 1, y = 0;
  for (int t = 0; t < 24; t++) {
    RHO[x + 5 * y] = (unsigned)(((t + 1) * (t + 2) / 2) % 64);
    int nx = y, ny = (2 * x + 3 * y) % 5;
    x = nx;
    y = ny;
  }
  /* iota (FIPS 202 3.2.5): RC[i] bit 2^j - 1 = rc(j + 7 i) for j = 0..6 */
  for (int i = 0; i < 24; i++) {
    uint64_t c = 0;
    for (int j = 0; j <= 6; j++)
      if (rc_bit(j + 7 * i)) c |= (uint64_t)1 << ((1u << j) - 1);
    RC[i] = c;
  }
  keccak_ready = 1;
}

static void keccak_f1600(uint64_t A[25]) {
  if (!keccak_ready) build_keccak();
  for (int round = 0; round < 24; round++) {
    /* theta */
    uint64_t C[5], D[5];
    for (int x = 0; x < 5; x++)
      C[x] = A[x] ^ A[x + 5] ^ A[x + 10] ^ A[x + 15] ^ A[x + 20];
    for (int x = 0; x < 5; x++)
      D[x] = C[(x + 4) % 5] ^ rotl64(C[(x + 1) % 5], 1);
    for (int x = 0; x < 5; x++)
      for (int y = 0; y < 5; y++) A[x + 5 * y] ^= D[x];
    /* rho and pi: B[y][2x+3y] = rot(A[x][y], r[x][y]) */
    uint64_t Bm[25];
    for (int x = 0; x < 5; x++)
      for (int y = 0; y < 5; y++)
        Bm[y + 5 * ((2 * x + 3 * y) % 5)] = rotl64(A[x + 5 * y], RHO[x + 5 * y]);
    /* chi */
    for (int x = 0; x < 5; x++)
      for (int y = 0; y < 5; y++)
        A[x + 5 * y] = Bm[x + 5 * y] ^
                       ((~Bm[(x + 1) % 5 + 5 * y]) & Bm[(x + 2) % 5 + 5 * y]);
    /* iota */
    A[0] ^= RC[round];
  }
}

/* SHA3-256 = Keccak[512](M || 01, 256): rate 136 bytes, pad10*1. */
void orc_sha3_256(const uint8_t *msg, size_t len, uint8_t out[32]) {
  const size_t rate = 136;
  uint64_t A[25];
  memset(A, 0, sizeof A);
  size_t nblocks = len / rate + 1;  /* the padded message */
  for (size_t blk = 0; blk < nblocks; blk++) {
    uint8_t block[136];
    memset(block, 0, rate);
    size_t off = blk * rate;
    size_t take = (off < len) ? ((len - off < rate) ? len - off : rate) : 0;
    if (take) memcpy(block, msg + off, take);
    if (blk == nblocks - 1) {
      block[take] ^= 0x06;        /* SHA-3 domain bits 01, then pad bit 1 */
      block[rate - 1] ^= 0x80;    /* final pad bit                        */
    }
    for (size_t i = 0; i < rate / 8; i++) {
      uint64_t lane = 0;
      for (int b = 0; b < 8; b++) lane |= (uint64_t)block[8 * i + b] << (8 * b);
      A[i] ^= lane;
    }
    keccak_f1600(A);
  }
  for (int i = 0; i < 32; i++) out[i] = (uint8_t)(A[i / 8] >> (8 * (i % 8)));
}

void orc_htree(const uint8_t *msg, size_t len, uint8_t out[32]) {
  size_t m = (len + ORC_TREE_CHUNK - 1) / ORC_TREE_CHUNK;
  if (m == 0) m = 1;
  uint8_t *leaves = (uint8_t *)malloc(32 * m);
  for (size_t i = 0; i < m; i++) {
    size_t off = i * ORC_TREE_CHUNK;
    size_t take = len - off < ORC_TREE_CHUNK ? len - off : ORC_TREE_CHUNK;
    if (off >= len) take = 0;
    orc_sha3_256(msg + off, take, leaves + 32 * i);
  }
  orc_sha3_256(leaves, 32 * m, out);
  free(leaves);
}

/* ======================================================================== */
/* Rounded-Gaussian CDF table and inverse sampler                            */
/* ======================================================================== */

static double phi(double x) { return 0.5 * (1.0 + erf(x / sqrt(2.0))); }

/* p(k) = Phi((k+1/2)/sigma) - Phi((k-1/2)/sigma) for |k| <= c, renormalised;
 * T[k] = round_half_up(2^15 * (p(0) + 2 sum_{j=1..k} p(j))) - 1. */
int orc_cdf_table(double sigma, uint32_t clip, uint16_t *T) {
  double p[16];
  double total = 0.0;
  for (uint32_t k = 0; k <= clip; k++) {
    p[k] = phi((k + 0.5) / sigma) - phi((k - 0.5) / sigma);
    total += (k == 0) ? p[k] : 2.0 * p[k];
  }
  double cum = 0.0;
  for (uint32_t k = 0; k < clip; k++) {
    cum += (k == 0) ? p[0] / total : 2.0 * p[k] / total;
    double v = floor(32768.0 * cum + 0.5) - 1.0;
    if (v < 0.0) v = 0.0;  /* rejected below if it breaks monotonicity */
    T[k] = (uint16_t)v;
  }
  for (uint32_t k = 1; k < clip; k++)
    if (T[k] <= T[k - 1]) return -1;
  if (clip > 0 && T[clip - 1] >= 32767) return -1;
  return 0;
}

/* word w: t = w >> 1, magnitude = #{i < c : t > T[i]}, sign = bit 0 */
int orc_sample(uint16_t w, const uint16_t *T, uint32_t clip) {
  unsigned t = w >> 1;
  int mag = 0;
  for (uint32_t i = 0; i < clip; i++)
    if (t > T[i]) mag++;
  return (w & 1) ? -mag : mag;
}

void orc_noise(const uint8_t key[16], uint64_t domain, const uint16_t *T,
               uint32_t clip, size_t count, int8_t *out) {
  uint8_t rk[176];
  orc_aes128_key_expand(key, rk);
  uint8_t blk[16];
  for (size_t k = 0; k < count; k++) {
    if (k % 8 == 0) orc_ctr_block(rk, domain, k / 8, blk);
    size_t w = k % 8;
    uint16_t word = (uint16_t)(blk[2 * w] | (blk[2 * w + 1] << 8));
    out[k] = (int8_t)orc_sample(word, T, clip);
  }
}

/* ======================================================================== */
/* Matrices                                                                  */
/* ======================================================================== */

void orc_expand_A(const uint8_t seedA[16], uint32_t n, uint32_t logq,
                  uint16_t *A) {
  uint8_t rk[176];
  orc_aes128_key_expand(seedA, rk);
  uint16_t mask = (uint16_t)((1u << logq) - 1u);
  uint8_t blk[16];
  for (uint32_t i = 0; i < n; i++) {
    for (uint32_t j = 0; j < n; j += 8) {
      uint64_t b = (uint64_t)i * (n / 8) + j / 8;
      orc_ctr_block(rk, 0, b, blk);
      for (int t = 0; t < 8; t++)
        A[(size_t)i * n + j + t] =
            (uint16_t)(blk[2 * t] | (blk[2 * t + 1] << 8)) & mask;
    }
  }
}

void orc_mul_AS(uint32_t n, uint32_t k, uint32_t logq, const uint16_t *A,
                const int8_t *St, const int8_t *E, uint16_t *out) {
  uint64_t mask = (1ull << logq) - 1ull;
  for (uint32_t i = 0; i < n; i++) {
    for (uint32_t c = 0; c < k; c++) {
      int64_t acc = E ? E[(size_t)i * k + c] : 0;
      for (uint32_t j = 0; j < n; j++)
        acc += (int64_t)A[(size_t)i * n + j] * St[(size_t)c * n + j];
      out[(size_t)i * k + c] = (uint16_t)((uint64_t)acc & mask);
    }
  }
}

void orc_mul_SA(uint32_t m, uint32_t n, uint32_t ncol, uint32_t logq,
                const int8_t *S, const uint16_t *X, const int8_t *E,
                uint16_t *out) {
  uint64_t mask = (1ull << logq) - 1ull;
  int64_t *acc = (int64_t *)malloc(sizeof(int64_t) * ncol);
  for (uint32_t r = 0; r < m; r++) {
    for (uint32_t j = 0; j < ncol; j++)
      acc[j] = E ? E[(size_t)r * ncol + j] : 0;
    /* acc[j] = sum_i S[r][i] X[i][j]: exact integer sum, accumulated row by
     * row of X */
    for (uint32_t i = 0; i < n; i++) {
      int64_t s = S[(size_t)r * n + i];
      const uint16_t *xrow = X + (size_t)i * ncol;
      for (uint32_t j = 0; j < ncol; j++) acc[j] += s * xrow[j];
    }
    for (uint32_t j = 0; j < ncol; j++)
      out[(size_t)r * ncol + j] = (uint16_t)((uint64_t)acc[j] & mask);
  }
  free(acc);
}

/* ======================================================================== */
/* KEM (Alg. 1-5)                                                            */
/* ======================================================================== */

size_t orc_pk_bytes(const orc_params *p) {
  return 16 + 2 * (size_t)p->n * p->nbar;
}
size_t orc_sk_bytes(const orc_params *p) {
  return (size_t)p->nbar * p->n + 32 + 32 + orc_pk_bytes(p);
}
size_t orc_ct_bytes(const orc_params *p) {
  return 2 * (size_t)p->mbar * p->n + 2 * (size_t)p->mbar * p->nbar;
}
size_t orc_mu_bytes(const orc_params *p) {
  return ((size_t)p->mbar * p->nbar * p->B + 7) / 8;
}

int orc_check_params(const orc_params *p) {
  if (p->n == 0 || p->n % 8 != 0) return -1;
  if (p->nbar != 8 || p->mbar != 8) return -1;
  if (p->logq < 2 || p->logq > 16) return -1;
  if (p->B < 1 || p->B > 4 || p->B >= p->logq) return -1;
  if (p->clip < 1 || p->clip > 15) return -1;
  if (!(p->sigma > 0.0)) return -1;
  uint16_t T[16];
  if (orc_cdf_table(p->sigma, p->clip, T) != 0) return -1;
  return 0;
}

static void put_u16le(uint8_t *dst, uint16_t v) {
  dst[0] = (uint8_t)v;
  dst[1] = (uint8_t)(v >> 8);
}
static uint16_t get_u16le(const uint8_t *src) {
  return (uint16_t)(src[0] | (src[1] << 8));
}

/* H(prefix || msg) for the short, domain-separated derivations */
static void sha3_prefixed(uint8_t prefix, const uint8_t *msg, size_t len,
                          uint8_t out[32]) {
  uint8_t *buf = (uint8_t *)malloc(len + 1);
  buf[0] = prefix;
  memcpy(buf + 1, msg, len);
  orc_sha3_256(buf, len + 1, out);
  free(buf);
}

/* KeyGen, Alg. 1 with S an n x nbar matrix:
 *   seedA = H(0x41 || ms)[0:16], seedSE = H(0x53 || ms)[0:16], z = H(0x5A || ms)
 *   A <- sample(seedA); S^T <- chi (domain 1); E <- chi (domain 2)
 *   B = A S + E mod q;  pk = seedA || B;  sk = S^T || z || H(pk) || pk */
int orc_keygen(const orc_params *p, const uint8_t ms[32], uint8_t *pk,
               uint8_t *sk, uint16_t *A_out) {
  if (orc_check_params(p)) return -1;
  uint32_t n = p->n, nb = p->nbar;
  uint16_t T[16];
  orc_cdf_table(p->sigma, p->clip, T);
  uint8_t h[32], seedA[16], seedSE[16], z[32];
  sha3_prefixed(0x41, ms, 32, h);
  memcpy(seedA, h, 16);
  sha3_prefixed(0x53, ms, 32, h);
  memcpy(seedSE, h, 16);
  sha3_prefixed(0x5A, ms, 32, z);

  uint16_t *A = A_out ? A_out : (uint16_t *)malloc(sizeof(uint16_t) * n * n);
  orc_expand_A(seedA, n, p->logq, A);
  int8_t *St = (int8_t *)malloc((size_t)nb * n);
  int8_t *E = (int8_t *)malloc((size_t)n * nb);
  orc_noise(seedSE, 1, T, p->clip, (size_t)nb * n, St);
  orc_noise(seedSE, 2, T, p->clip, (size_t)n * nb, E);
  uint16_t *Bm = (uint16_t *)malloc(sizeof(uint16_t) * n * nb);
  orc_mul_AS(n, nb, p->logq, A, St, E, Bm);

  memcpy(pk, seedA, 16);
  for (size_t i = 0; i < (size_t)n * nb; i++) put_u16le(pk + 16 + 2 * i, Bm[i]);
  size_t pkb = orc_pk_bytes(p);
  uint8_t *q = sk;
  memcpy(q, St, (size_t)nb * n);
  q += (size_t)nb * n;
  memcpy(q, z, 32);
  q += 32;
  orc_htree(pk, pkb, q);
  q += 32;
  memcpy(q, pk, pkb);

  free(Bm);
  free(E);
  free(St);
  if (!A_out) free(A);
  return 0;
}

/* Encrypt, Alg. 2 with r stacked into S' (mbar x n), derandomised by
 * seedSE' so that Decaps can recompute it (Alg. 5):
 *   S' (domain 3), E' (domain 4), E'' (domain 5) from seedSE'
 *   B' = S' A + E';  V = S' B + E'';  C = V + Enc(mu);  c = B' || C */
static void encrypt(const orc_params *p, const uint8_t *pk, const uint16_t *A,
                    const uint8_t *mu, const uint8_t seed_se[16], uint8_t *ct,
                    orc_trace *tr) {
  uint32_t n = p->n, nb = p->nbar, mb = p->mbar, D = p->logq, Bb = p->B;
  uint16_t T[16];
  orc_cdf_table(p->sigma, p->clip, T);
  uint16_t *Aloc = NULL;
  if (!A) {
    Aloc = (uint16_t *)malloc(sizeof(uint16_t) * n * n);
    orc_expand_A(pk, n, D, Aloc);
    A = Aloc;
  }
  int8_t *Sp = (int8_t *)malloc((size_t)mb * n);
  int8_t *Ep = (int8_t *)malloc((size_t)mb * n);
  int8_t Epp[64];
  orc_noise(seed_se, 3, T, p->clip, (size_t)mb * n, Sp);
  orc_noise(seed_se, 4, T, p->clip, (size_t)mb * n, Ep);
  orc_noise(seed_se, 5, T, p->clip, (size_t)mb * nb, Epp);

  uint16_t *Bp = (uint16_t *)malloc(sizeof(uint16_t) * mb * n);
  orc_mul_SA(mb, n, n, D, Sp, A, Ep, Bp);

  uint16_t *Bm = (uint16_t *)malloc(sizeof(uint16_t) * n * nb);
  for (size_t i = 0; i < (size_t)n * nb; i++) Bm[i] = get_u16le(pk + 16 + 2 * i);
  uint16_t V[64];
  orc_mul_SA(mb, n, nb, D, Sp, Bm, Epp, V);

  uint32_t qmask = (1u << D) - 1u;
  for (uint32_t r = 0; r < mb; r++) {
    for (uint32_t l = 0; l < nb; l++) {
      uint32_t sym = 0;
      for (uint32_t u = 0; u < Bb; u++) {
        uint32_t bit = (r * nb + l) * Bb + u;
        sym |= (uint32_t)((mu[bit / 8] >> (bit % 8)) & 1) << u;
      }
      uint32_t c = (V[r * nb + l] + (sym << (D - Bb))) & qmask;  /* Enc */
      V[r * nb + l] = (uint16_t)c;
    }
  }
  for (size_t i = 0; i < (size_t)mb * n; i++) put_u16le(ct + 2 * i, Bp[i]);
  for (size_t i = 0; i < (size_t)mb * nb; i++)
    put_u16le(ct + 2 * (size_t)mb * n + 2 * i, V[i]);

  if (tr) {
    if (tr->Sp) memcpy(tr->Sp, Sp, (size_t)mb * n);
    if (tr->Ep) memcpy(tr->Ep, Ep, (size_t)mb * n);
    if (tr->Epp) memcpy(tr->Epp, Epp, (size_t)mb * nb);
  }
  free(Bm);
  free(Bp);
  free(Ep);
  free(Sp);
  free(Aloc);
}

/* K' = H(H(pk) || mu) and seedSE' = H(0x01 || H(pk) || mu)[0:16] */
static void derive(const orc_params *p, const uint8_t pkh[32],
                   const uint8_t *mu, uint8_t kprime[32],
                   uint8_t seed_se[16]) {
  size_t mub = orc_mu_bytes(p);
  uint8_t buf[1 + 32 + 32];
  memcpy(buf, pkh, 32);
  memcpy(buf + 32, mu, mub);
  orc_sha3_256(buf, 32 + mub, kprime);
  uint8_t h[32];
  sha3_prefixed(0x01, buf, 32 + mub, h);
  memcpy(seed_se, h, 16);
}

/* Encaps, Alg. 4:  mu = H(0x4D || coins)[0 : B*mbar*nbar/8];
 * c = Encrypt(pk, mu);  K' = H(H(pk) || mu);  K = H(K' || H(c)) */
int orc_encaps_trace(const orc_params *p, const uint8_t *pk, const uint16_t *A,
                     const uint8_t coins[32], uint8_t *ct, uint8_t K[32],
                     orc_trace *tr) {
  if (orc_check_params(p)) return -1;
  uint8_t h[32], mu[32], pkh[32], kprime[32], seed_se[16], hc[32];
  sha3_prefixed(0x4D, coins, 32, h);
  memset(mu, 0, sizeof mu);
  memcpy(mu, h, orc_mu_bytes(p));
  orc_htree(pk, orc_pk_bytes(p), pkh);
  derive(p, pkh, mu, kprime, seed_se);
  encrypt(p, pk, A, mu, seed_se, ct, tr);
  orc_htree(ct, orc_ct_bytes(p), hc);
  uint8_t buf[64];
  memcpy(buf, kprime, 32);
  memcpy(buf + 32, hc, 32);
  orc_sha3_256(buf, 64, K);
  if (tr) {
    memcpy(tr->mu, mu, 32);
    memcpy(tr->pkh, pkh, 32);
    memcpy(tr->kprime, kprime, 32);
    memcpy(tr->seed_se, seed_se, 16);
    memcpy(tr->hc, hc, 32);
  }
  return 0;
}

int orc_encaps(const orc_params *p, const uint8_t *pk, const uint16_t *A,
               const uint8_t coins[32], uint8_t *ct, uint8_t K[32]) {
  return orc_encaps_trace(p, pk, A, coins, ct, K, NULL);
}

/* Decaps, Alg. 5 with Decrypt of Alg. 3:
 *   M = C - B' S;  mu' = Dec(M), Dec(x) = ((x + 2^(D-B-1)) >> (D-B)) mod 2^B
 *   c' = Encrypt(pk, mu');  K' = H(H(pk) || mu')
 *   K = H(K' || H(c)) if c' = c, else H(z || H(c)), selected without a
 *   data-dependent branch (implicit rejection). */
int orc_decaps_trace(const orc_params *p, const uint8_t *sk, const uint16_t *A,
                     const uint8_t *ct, uint8_t K[32], orc_trace *tr) {
  if (orc_check_params(p)) return -1;
  uint32_t n = p->n, nb = p->nbar, mb = p->mbar, D = p->logq, Bb = p->B;
  const int8_t *St = (const int8_t *)sk;
  const uint8_t *z = sk + (size_t)nb * n;
  const uint8_t *pkh = z + 32;
  const uint8_t *pk = pkh + 32;
  size_t ctb = orc_ct_bytes(p);
  uint32_t qmask = (1u << D) - 1u;

  uint16_t M[64];
  for (uint32_t r = 0; r < mb; r++) {
    for (uint32_t l = 0; l < nb; l++) {
      int64_t acc = get_u16le(ct + 2 * (size_t)mb * n + 2 * (r * nb + l));
      for (uint32_t j = 0; j < n; j++)
        acc -= (int64_t)get_u16le(ct + 2 * ((size_t)r * n + j)) *
               St[(size_t)l * n + j];
      M[r * nb + l] = (uint16_t)((uint64_t)acc & qmask);
    }
  }
  uint8_t mu[32];
  memset(mu, 0, sizeof mu);
  for (uint32_t r = 0; r < mb; r++) {
    for (uint32_t l = 0; l < nb; l++) {
      uint32_t x = M[r * nb + l];
      uint32_t sym = ((x + (1u << (D - Bb - 1))) >> (D - Bb)) & ((1u << Bb) - 1u);
      for (uint32_t u = 0; u < Bb; u++) {
        uint32_t bit = (r * nb + l) * Bb + u;
        mu[bit / 8] |= (uint8_t)(((sym >> u) & 1) << (bit % 8));
      }
    }
  }
  uint8_t kprime[32], seed_se[16], hc[32];
  derive(p, pkh, mu, kprime, seed_se);
  uint8_t *ct2 = (uint8_t *)malloc(ctb);
  encrypt(p, pk, A, mu, seed_se, ct2, NULL);
  orc_htree(ct, ctb, hc);
  uint8_t diff = 0;
  for (size_t i = 0; i < ctb; i++) diff |= ct[i] ^ ct2[i];
  /* eq_mask = 0xFF when diff == 0, else 0x00, computed without a branch */
  uint8_t eq_mask = (uint8_t)(((uint32_t)diff - 1u) >> 8);
  uint8_t buf[64];
  for (int i = 0; i < 32; i++)
    buf[i] = (uint8_t)((kprime[i] & eq_mask) | (z[i] & (uint8_t)~eq_mask));
  memcpy(buf + 32, hc, 32);
  orc_sha3_256(buf, 64, K);
  if (tr) {
    memcpy(tr->mu, mu, 32);
    memcpy(tr->pkh, pkh, 32);
    memcpy(tr->kprime, kprime, 32);
    memcpy(tr->seed_se, seed_se, 16);
    memcpy(tr->hc, hc, 32);
    if (tr->M) memcpy(tr->M, M, sizeof(uint16_t) * mb * nb);
    tr->eq = eq_mask ? 1 : 0;
  }
  free(ct2);
  return 0;
}

int orc_decaps(const orc_params *p, const uint8_t *sk, const uint16_t *A,
               const uint8_t *ct, uint8_t K[32]) {
  return orc_decaps_trace(p, sk, A, ct, K, NULL);
}

/* ---- batches: independent items, optionally spread over threads ------- */

/* the lazily built tables must exist before threads share them */
static void init_tables(void) {
  if (!sbox_ready) build_sbox();
  if (!keccak_ready) build_keccak();
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int orc_keygen_batch(const orc_params *p, const uint8_t *ms, size_t count,
                     uint8_t *pk, uint8_t *sk, int nthreads) {
  if (orc_check_params(p)) return -1;
  init_tables();
  size_t pkb = orc_pk_bytes(p), skb = orc_sk_bytes(p);
  long long cnt = (long long)count;
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long i = 0; i < cnt; i++)
    orc_keygen(p, ms + 32 * i, pk + pkb * i, sk + skb * i, NULL);
  return 0;
}

int orc_encaps_batch(const orc_params *p, const uint8_t *pk, const uint16_t *A,
                     const uint8_t *coins, size_t count, uint8_t *ct,
                     uint8_t *K, int nthreads) {
  if (orc_check_params(p)) return -1;
  init_tables();
  size_t ctb = orc_ct_bytes(p);
  long long cnt = (long long)count;
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long i = 0; i < cnt; i++)
    orc_encaps(p, pk, A, coins + 32 * i, ct + ctb * i, K + 32 * i);
  return 0;
}

int orc_decaps_batch(const orc_params *p, const uint8_t *sk, const uint16_t *A,
                     const uint8_t *ct, size_t count, uint8_t *K,
                     int nthreads) {
  if (orc_check_params(p)) return -1;
  init_tables();
  size_t ctb = orc_ct_bytes(p);
  long long cnt = (long long)count;
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long i = 0; i < cnt; i++)
    orc_decaps(p, sk, A, ct + ctb * i, K + 32 * i);
  return 0;
}
