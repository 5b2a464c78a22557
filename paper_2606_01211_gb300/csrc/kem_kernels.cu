// kem_kernels.cu -- CUDA-core kernels of the plain-LWE KEM hot path (sm_103a).
//
//   k_expand_A      sample(seedA) of Alg. 1: AES-128-CTR expansion of A,
//                   16-byte coalesced stores.
//   k_noise         the error/secret distributions of Alg. 1-2 (Tab. 1:
//                   rounded Gaussian) by CDF-table inverse sampling of AES
//                   counter streams.
//   k_mul_as        B = A S + E of Alg. 1 (A stored or regenerated).
//   k_decrypt       M = C - B' S and mu' = Dec(M) of Alg. 3.
//   k_mul_sa        B' = S' A + E' of Alg. 2, one encryption per CTA row,
//                   stored A; with a compare epilogue for Alg. 5.
//   k_mul_sa_fused  the same with A regenerated from its seed in-CTA.
//   k_v_encode      V = S' B + E'', C = V + Enc(mu) of Alg. 2 (or compare).
//   k_keygen_seeds, k_derive, k_tree, k_final_key: the hashing of
//                   Alg. 4-5 (SHA3-256) and the Fujisaki-Okamoto selection.
#include <cuda_bf16.h>

#include <algorithm>

#include "aes.cuh"
#include "common.cuh"
#include "gemm_tc.h"
#include "kem_kernels.h"
#include "keccak.cuh"

// The round table T0 (see aes.cuh); written by lwe_upload_aes_table.
__device__ uint32_t g_aes_T0[256];

// ---------------------------------------------------------------------------
// A expansion: thread per 16-byte block, grid-stride; one key per grid.y.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512, 1) k_expand_A(const uint8_t *__restrict__ seeds,
                                                  uint32_t seed_stride, uint32_t n,
                                                  uint32_t logq, uint16_t *__restrict__ A,
                                                  uint64_t a_stride) {
  extern __shared__ uint32_t sT[];
  aes_fill_smem(sT, g_aes_T0);
  __syncthreads();
  const AesTab tab = aes_tab(sT);
  const uint32_t e = blockIdx.y;
  uint32_t key[4], rk[44];
  aes_load_key(seeds + (size_t)e * seed_stride, key);
  aes_key_expand(tab, key, rk);
  const uint32_t m = (1u << logq) - 1u;
  const uint32_t mm = m | (m << 16);
  const uint64_t nblk = (uint64_t)n * n / 8;
  uint4 *out = reinterpret_cast<uint4 *>(A + (size_t)e * a_stride);
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk;
       b += (uint64_t)gridDim.x * blockDim.x) {
    uint4 v = aes_ctr_block(tab, rk, 0, b);
    v.x &= mm;
    v.y &= mm;
    v.z &= mm;
    v.w &= mm;
    out[b] = v;
  }
}

// ---------------------------------------------------------------------------
// Noise: a warp generates one run of NOISE_RUN counter blocks of one stream
// of one item (4 blocks per lane, two at a time, contiguous stores).
// Sampling (Tab. 1, rounded Gaussian by CDF inversion): a 16-bit word w gives
// t = w >> 1, |e| = #{i : t > T[i]}, e < 0 iff w & 1.  Every CTA first
// tabulates e for all 65536 words in shared memory (64 KB of int8), so a
// sample costs one byte load; the table is built from T with the same
// comparison rule.
// ---------------------------------------------------------------------------
#define NOISE_TAB_OFF AES_SMEM_BYTES
#define NOISE_SMEM_BYTES (AES_SMEM_BYTES + 65536)

LWE_DEV int cdf_mag(uint32_t t, const NoiseArgs &a) {
  int mag = 0;
#pragma unroll
  for (int i = 0; i < 15; i++) mag += (t > a.T[i]) ? 1 : 0;
  return mag;
}

LWE_DEV void noise_fill_table(uint32_t *tab, const NoiseArgs &a) {
  // word j holds the samples of w = 4j .. 4j+3 (t = 2j, 2j, 2j+1, 2j+1)
  for (uint32_t j = threadIdx.x; j < 16384; j += blockDim.x) {
    const int m0 = cdf_mag(2 * j, a), m1 = cdf_mag(2 * j + 1, a);
    tab[j] = (uint32_t)(m0 & 0xff) | ((uint32_t)(-m0 & 0xff) << 8) | ((uint32_t)(m1 & 0xff) << 16) |
             ((uint32_t)(-m1 & 0xff) << 24);
  }
}

LWE_DEV int tab_sample(const char *smem, uint32_t w16) {
  return *reinterpret_cast<const int8_t *>(smem + NOISE_TAB_OFF + w16);
}

LWE_DEV void noise_store(const char *smem, const NoiseOut &o, uint8_t *base, uint32_t b, uint4 v) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  int smp[8];
#pragma unroll
  for (int t = 0; t < 4; t++) {
    smp[2 * t] = tab_sample(smem, w[t] & 0xffffu);
    smp[2 * t + 1] = tab_sample(smem, w[t] >> 16);
  }
  const bool full = (8 * b + 8 <= o.nsamples);
  if (o.fmt == NOISE_I8) {
    if (full) {
      const uint32_t lo = __byte_perm(__byte_perm(smp[0], smp[1], 0x0040),
                                      __byte_perm(smp[2], smp[3], 0x0040), 0x5410);
      const uint32_t hi = __byte_perm(__byte_perm(smp[4], smp[5], 0x0040),
                                      __byte_perm(smp[6], smp[7], 0x0040), 0x5410);
      *reinterpret_cast<uint2 *>(base + 8 * (size_t)b) = make_uint2(lo, hi);
    } else {
      for (int t = 0; t < 8; t++)
        if (8 * b + t < o.nsamples) base[8 * (size_t)b + t] = (uint8_t)(int8_t)smp[t];
    }
  } else {  // bf16: small integers are exact
    __nv_bfloat16 *bp = reinterpret_cast<__nv_bfloat16 *>(base);
    if (full) {
      uint32_t pk[4];
#pragma unroll
      for (int t = 0; t < 4; t++) {
        __nv_bfloat162 h2 = __floats2bfloat162_rn((float)smp[2 * t], (float)smp[2 * t + 1]);
        pk[t] = *reinterpret_cast<uint32_t *>(&h2);
      }
      *reinterpret_cast<uint4 *>(bp + 8 * (size_t)b) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    } else {
      for (int t = 0; t < 8; t++)
        if (8 * b + t < o.nsamples) bp[8 * (size_t)b + t] = __float2bfloat16_rn((float)smp[t]);
    }
  }
}

__global__ void __launch_bounds__(512, 1) k_noise(NoiseArgs a) {
  extern __shared__ uint32_t sT[];
  aes_fill_smem(sT, g_aes_T0);
  noise_fill_table(sT + NOISE_TAB_OFF / 4, a);
  __syncthreads();
  const AesTab tab = aes_tab(sT);
  const char *smem = reinterpret_cast<const char *>(sT);
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nruns = (uint64_t)a.count * a.runs_per_item;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t run = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); run < nruns;
       run += nwarps) {
    const uint32_t e = (uint32_t)(run / a.runs_per_item);
    uint32_t r = (uint32_t)(run % a.runs_per_item);
    uint32_t s = 0;
    while (s + 1 < a.nout && r >= a.out[s].runs) {
      r -= a.out[s].runs;
      s++;
    }
    const NoiseOut o = a.out[s];
    uint32_t rk[44];
    const uint4 *rkp = reinterpret_cast<const uint4 *>(a.rk + 44 * (size_t)e);
#pragma unroll
    for (int i = 0; i < 11; i++) {
      const uint4 v = __ldg(rkp + i);
      rk[4 * i] = v.x;
      rk[4 * i + 1] = v.y;
      rk[4 * i + 2] = v.z;
      rk[4 * i + 3] = v.w;
    }
    const uint32_t nblk = (o.nsamples + 7) / 8;
    uint8_t *base = reinterpret_cast<uint8_t *>(o.base) + (size_t)e * o.item_stride;
    const uint32_t b0 = r * NOISE_RUN + lane;
    if (r * NOISE_RUN + NOISE_RUN <= nblk) {
      // full run: two independent blocks in flight per lane
#pragma unroll
      for (uint32_t j = 0; j < NOISE_RUN / 32; j += 2) {
        const uint32_t ba = b0 + 32 * j, bb = ba + 32;
        const uint4 va = aes_ctr_block(tab, rk, o.domain, ba);
        const uint4 vb = aes_ctr_block(tab, rk, o.domain, bb);
        noise_store(smem, o, base, ba, va);
        noise_store(smem, o, base, bb, vb);
      }
    } else {
#pragma unroll 1
      for (uint32_t b = b0; b < nblk; b += 32) noise_store(smem, o, base, b, aes_ctr_block(tab, rk, o.domain, b));
    }
  }
}

// ---------------------------------------------------------------------------
// Rows times S^T: out[r][l] = sum_j X[r][j] * St[l][j] for l < 8.
// A warp owns a row; a lane takes 8-element chunks (16 bytes of X, one AES
// block when X = A is regenerated) and uses dp2a: two 16-bit entries of X
// (as signed halves, the same residues mod 2^16) times two int8 of S^T.
// ---------------------------------------------------------------------------
LWE_DEV void dot8_chunk(const uint4 x, const int8_t *__restrict__ St, uint32_t n,
                        uint32_t j, int acc[8]) {
#pragma unroll
  for (int l = 0; l < 8; l++) {
    const uint2 s = ld_nc_u2(St + (size_t)l * n + j);
    acc[l] = __dp2a_lo((int)x.x, (int)s.x, acc[l]);
    acc[l] = __dp2a_hi((int)x.y, (int)s.x, acc[l]);
    acc[l] = __dp2a_lo((int)x.z, (int)s.y, acc[l]);
    acc[l] = __dp2a_hi((int)x.w, (int)s.y, acc[l]);
  }
}

LWE_DEV void warp_allreduce8(int acc[8]) {
#pragma unroll
  for (int l = 0; l < 8; l++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], o);
  }
}

template <bool FUSED>
__global__ void __launch_bounds__(256) k_mul_as(MulAsArgs a) {
  extern __shared__ uint32_t sT[];
  AesTab tab;
  uint32_t rk[44];
  const uint32_t e = blockIdx.y;
  if (FUSED) {
    aes_fill_smem(sT, g_aes_T0);
    __syncthreads();
    tab = aes_tab(sT);
    uint32_t key[4];
    aes_load_key(a.seeds + (size_t)e * a.seed_stride, key);
    aes_key_expand(tab, key, rk);
  }
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t i = blockIdx.x * 8 + warp;
  if (i >= a.n) return;
  const uint32_t n = a.n;
  const int8_t *St = a.St + (size_t)e * a.st_stride;
  int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const uint16_t *Arow = FUSED ? nullptr : a.A + (size_t)e * a.a_stride + (size_t)i * n;
  for (uint32_t jc = lane; jc < n / 8; jc += 32) {
    uint4 x;
    if (FUSED)
      x = aes_ctr_block(tab, rk, 0, (uint64_t)i * (n / 8) + jc);
    else
      x = ld_nc_u4(Arow + 8 * (size_t)jc);
    if (FUSED) {
      const uint32_t m = (1u << a.logq) - 1u, mm = m | (m << 16);
      x.x &= mm;
      x.y &= mm;
      x.z &= mm;
      x.w &= mm;
    }
    dot8_chunk(x, St, n, 8 * jc, acc);
  }
  warp_allreduce8(acc);
  if (lane == 0) {
    const uint32_t m = (1u << a.logq) - 1u;
    uint32_t v[8];
    const int8_t *E = a.E ? a.E + (size_t)e * a.e_stride + (size_t)i * 8 : nullptr;
#pragma unroll
    for (int l = 0; l < 8; l++) v[l] = (uint32_t)(acc[l] + (E ? (int)E[l] : 0)) & m;
    const uint4 pk = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16),
                                v[6] | (v[7] << 16));
    *reinterpret_cast<uint4 *>(a.out + (size_t)e * a.out_stride + 16 * (size_t)i) = pk;
    if (a.out2)
      *reinterpret_cast<uint4 *>(a.out2 + (size_t)e * a.out2_stride + 16 * (size_t)i) = pk;
  }
}

// Decrypt (Alg. 3): warp r of CTA e computes row r of M = C - B' S and the
// B message bits of its eight coefficients.
__global__ void __launch_bounds__(256) k_decrypt(DecryptArgs a) {
  const uint32_t e = blockIdx.x;
  const uint32_t r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = a.n;
  const uint8_t *ct = a.ct + (size_t)e * a.ct_bytes;
  const uint16_t *Brow = reinterpret_cast<const uint16_t *>(ct) + (size_t)r * n;
  const int8_t *St = a.sk_ptrs ? reinterpret_cast<const int8_t *>(a.sk_ptrs[e]) : a.St;
  int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // up to four 16-byte chunks of the row per lane are requested together,
  // so a warp waits for one memory latency per 2048 bytes, not per chunk
  const uint32_t nch = n / 8;
  for (uint32_t base = 0; base < nch; base += 128) {
    uint4 x[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t jc = base + lane + 32 * k;
      x[k] = jc < nch ? ld_nc_u4(Brow + 8 * (size_t)jc) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t jc = base + lane + 32 * k;
      if (jc < nch) dot8_chunk(x[k], St, n, 8 * jc, acc);
    }
  }
  warp_allreduce8(acc);
  if (lane == 0) {
    const uint32_t D = a.logq, Bb = a.B, m = (1u << D) - 1u;
    const uint16_t *C = reinterpret_cast<const uint16_t *>(ct + 16 * (size_t)n) + 8 * r;
    uint32_t bits = 0;
#pragma unroll
    for (int l = 0; l < 8; l++) {
      const uint32_t M = ((uint32_t)C[l] - (uint32_t)acc[l]) & m;
      const uint32_t sym = ((M + (1u << (D - Bb - 1))) >> (D - Bb)) & ((1u << Bb) - 1u);
      bits |= sym << (l * Bb);
    }
    uint8_t *mu = a.mu + (size_t)e * 32 + r * Bb;
    for (uint32_t t = 0; t < Bb; t++) mu[t] = (uint8_t)(bits >> (8 * t));
  }
}

// ---------------------------------------------------------------------------
// S' A (+ E') with stored A.  CTA (column block of 64, item e); warp w takes
// rows i = w (mod 8); lane l takes columns j0 + 2l, j0 + 2l + 1.
// ---------------------------------------------------------------------------
#define SA_CH 512

template <bool CMP>
__global__ void __launch_bounds__(256) k_mul_sa(MulSaArgs a) {
  __shared__ int4 sS[SA_CH][2];  // S'[0..7][i] for a chunk of rows
  const uint32_t e = blockIdx.y, j0 = blockIdx.x * 64;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = a.n;
  const int8_t *S = a.S + (size_t)e * a.s_stride;
  const uint16_t *Aitem = a.A_ptrs ? a.A_ptrs[e] : a.A;
  const uint32_t j = j0 + 2 * lane;
  const bool jvalid = j < n;
  int acc[8][2];
#pragma unroll
  for (int k = 0; k < 8; k++) acc[k][0] = acc[k][1] = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += SA_CH) {
    __syncthreads();
    for (uint32_t idx = threadIdx.x; idx < SA_CH * 8; idx += blockDim.x) {
      const uint32_t k = idx / SA_CH, ii = idx % SA_CH;
      const int v = (i0 + ii < n) ? (int)S[(size_t)k * n + i0 + ii] : 0;
      reinterpret_cast<int *>(&sS[ii][0])[k] = v;
    }
    __syncthreads();
    const uint32_t rows = min((uint32_t)SA_CH, n - i0);
    for (uint32_t ii = warp; ii < rows; ii += 8) {
      uint32_t av = 0;
      if (jvalid) av = __ldg(reinterpret_cast<const uint32_t *>(Aitem + (size_t)(i0 + ii) * n + j));
      const int x0 = (int)(av & 0xffffu), x1 = (int)(av >> 16);
      const int4 s0 = sS[ii][0], s1 = sS[ii][1];
      const int s[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
      for (int k = 0; k < 8; k++) {
        acc[k][0] += s[k] * x0;
        acc[k][1] += s[k] * x1;
      }
    }
  }
  // reduce the 8 warps' partial sums
  __syncthreads();
  int *red = reinterpret_cast<int *>(&sS[0][0]);  // [8 warps][16][32 lanes]
#pragma unroll
  for (int k = 0; k < 8; k++) {
    red[(warp * 16 + 2 * k + 0) * 32 + lane] = acc[k][0];
    red[(warp * 16 + 2 * k + 1) * 32 + lane] = acc[k][1];
  }
  __syncthreads();
  {
    const uint32_t k = warp;  // thread (k, lane) finishes row k, columns j, j+1
    int v0 = 0, v1 = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
      v0 += red[(w * 16 + 2 * k + 0) * 32 + lane];
      v1 += red[(w * 16 + 2 * k + 1) * 32 + lane];
    }
    const uint32_t m = (1u << a.logq) - 1u;
    uint32_t diff = 0;
    if (jvalid) {
      if (a.E) {
        const int8_t *E = a.E + (size_t)e * a.e_stride + (size_t)k * n + j;
        v0 += E[0];
        v1 += E[1];
      }
      const uint32_t packed = ((uint32_t)v0 & m) | (((uint32_t)v1 & m) << 16);
      uint32_t *o = reinterpret_cast<uint32_t *>(a.out + (size_t)e * a.out_stride +
                                                 2 * ((size_t)k * n + j));
      if (CMP)
        diff = packed ^ *o;
      else
        *o = packed;
    }
    if (CMP) {
      diff = __reduce_or_sync(0xffffffffu, diff);
      if (lane == 0 && diff) atomicOr(a.flags + e, 1u);
    }
  }
}

// S' A (+ E') with A regenerated: thread (column block cb of 8 columns,
// row slice rs of 32) generates A[i][j0+8cb .. +7] with one AES block per row.
template <bool CMP>
__global__ void __launch_bounds__(256) k_mul_sa_fused(MulSaArgs a) {
  extern __shared__ uint32_t smem[];
  uint32_t *sT = smem;                                           // 32 KB
  int4 *sS = reinterpret_cast<int4 *>(smem + AES_TABLE_WORDS);  // [SA_CH][2]
  aes_fill_smem(sT, g_aes_T0);
  __syncthreads();
  const AesTab tab = aes_tab(sT);
  const uint32_t e = blockIdx.y, j0 = blockIdx.x * 64;
  uint32_t key[4], rk[44];
  aes_load_key(a.seed_ptrs ? a.seed_ptrs[e] + a.seed_off : a.seedA, key);
  aes_key_expand(tab, key, rk);

  const uint32_t cb = threadIdx.x & 7, rs = threadIdx.x >> 3;
  const uint32_t n = a.n;
  const uint32_t mq = (1u << a.logq) - 1u, mm = mq | (mq << 16);
  const int8_t *S = a.S + (size_t)e * a.s_stride;
  const uint32_t jb = j0 + 8 * cb;
  const bool jvalid = jb < n;
  int acc[8][8];
#pragma unroll
  for (int k = 0; k < 8; k++)
#pragma unroll
    for (int c = 0; c < 8; c++) acc[k][c] = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += SA_CH) {
    __syncthreads();
    for (uint32_t idx = threadIdx.x; idx < SA_CH * 8; idx += blockDim.x) {
      const uint32_t k = idx / SA_CH, ii = idx % SA_CH;
      const int v = (i0 + ii < n) ? (int)S[(size_t)k * n + i0 + ii] : 0;
      reinterpret_cast<int *>(&sS[2 * ii])[k] = v;
    }
    __syncthreads();
    const uint32_t rows = min((uint32_t)SA_CH, n - i0);
    if (jvalid) {
      for (uint32_t ii = rs; ii < rows; ii += 32) {
        const uint4 v = aes_ctr_block(tab, rk, 0, (uint64_t)(i0 + ii) * (n / 8) + jb / 8);
        const uint32_t w[4] = {v.x & mm, v.y & mm, v.z & mm, v.w & mm};
        const int4 s0 = sS[2 * ii], s1 = sS[2 * ii + 1];
        const int s[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
        for (int c = 0; c < 8; c++) {
          const int x = (int)((w[c >> 1] >> (16 * (c & 1))) & 0xffffu);
#pragma unroll
          for (int k = 0; k < 8; k++) acc[k][c] += s[k] * x;
        }
      }
    }
  }
  // reduce over the 4 row slices inside a warp (lanes l, l^8, l^16, l^24)
#pragma unroll
  for (int k = 0; k < 8; k++)
#pragma unroll
    for (int c = 0; c < 8; c++) {
      acc[k][c] += __shfl_xor_sync(0xffffffffu, acc[k][c], 8);
      acc[k][c] += __shfl_xor_sync(0xffffffffu, acc[k][c], 16);
    }
  __syncthreads();
  int *red = reinterpret_cast<int *>(sS);  // [8 warps][8 cb][64]
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane < 8) {
#pragma unroll
    for (int k = 0; k < 8; k++)
#pragma unroll
      for (int c = 0; c < 8; c++) red[(warp * 8 + lane) * 64 + k * 8 + c] = acc[k][c];
  }
  __syncthreads();
  {
    // thread (k = warp, lane) finishes row k, columns j0 + 2 lane, +1
    const uint32_t k = warp;
    const uint32_t j = j0 + 2 * lane;
    const uint32_t cbj = (2 * lane) / 8, c0 = (2 * lane) % 8;
    int v0 = 0, v1 = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
      v0 += red[(w * 8 + cbj) * 64 + k * 8 + c0];
      v1 += red[(w * 8 + cbj) * 64 + k * 8 + c0 + 1];
    }
    uint32_t diff = 0;
    if (j < n) {
      if (a.E) {
        const int8_t *E = a.E + (size_t)e * a.e_stride + (size_t)k * n + j;
        v0 += E[0];
        v1 += E[1];
      }
      const uint32_t packed = ((uint32_t)v0 & mq) | (((uint32_t)v1 & mq) << 16);
      uint32_t *o = reinterpret_cast<uint32_t *>(a.out + (size_t)e * a.out_stride +
                                                 2 * ((size_t)k * n + j));
      if (CMP)
        diff = packed ^ *o;
      else
        *o = packed;
    }
    if (CMP) {
      diff = __reduce_or_sync(0xffffffffu, diff);
      if (lane == 0 && diff) atomicOr(a.flags + e, 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// V = S' B + E'' and C = V + Enc(mu) (Alg. 2); CTA per item, warp per row k.
// ---------------------------------------------------------------------------
template <bool CMP>
__global__ void __launch_bounds__(256) k_v_encode(VEncArgs a) {
  const uint32_t e = blockIdx.x;
  const uint32_t k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = a.n;
  const int8_t *S = a.S + (size_t)e * a.s_stride + (size_t)k * n;
  const uint8_t *pk = a.pk_ptrs ? a.pk_ptrs[e] + a.pk_off : a.pk;
  const uint16_t *Bm = reinterpret_cast<const uint16_t *>(pk + 16);
  int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (uint32_t i = lane; i < n; i += 32) {
    const int s = S[i];
    const uint4 b = ld_nc_u4(Bm + 8 * (size_t)i);
    const uint32_t w[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int l = 0; l < 8; l++) acc[l] += s * (int)((w[l >> 1] >> (16 * (l & 1))) & 0xffffu);
  }
  warp_allreduce8(acc);
  if (lane == 0) {
    const uint32_t D = a.logq, Bb = a.B, m = (1u << D) - 1u;
    const int8_t *Epp = a.Epp + (size_t)e * a.epp_stride + 8 * k;
    const uint8_t *mu = a.mu + (size_t)e * 32 + k * Bb;
    uint32_t bits = 0;
    for (uint32_t t = 0; t < Bb; t++) bits |= (uint32_t)mu[t] << (8 * t);
    uint32_t c[8];
#pragma unroll
    for (int l = 0; l < 8; l++) {
      const uint32_t sym = (bits >> (l * Bb)) & ((1u << Bb) - 1u);
      c[l] = ((uint32_t)(acc[l] + Epp[l]) + (sym << (D - Bb))) & m;
    }
    const uint4 pk = make_uint4(c[0] | (c[1] << 16), c[2] | (c[3] << 16), c[4] | (c[5] << 16),
                                c[6] | (c[7] << 16));
    uint4 *dst = reinterpret_cast<uint4 *>(a.ct + (size_t)e * a.ct_bytes + 16 * (size_t)n + 16 * k);
    if (CMP) {
      const uint4 old = *dst;
      const uint32_t diff = (old.x ^ pk.x) | (old.y ^ pk.y) | (old.z ^ pk.z) | (old.w ^ pk.w);
      if (diff) atomicOr(a.flags + e, 1u);
    } else {
      *dst = pk;
    }
  }
}

// ---------------------------------------------------------------------------
// Hashing: seeds (Alg. 1), derivation of K' and seedSE' (Alg. 4-5), tree
// hash of pk / c, and the final keys.
// ---------------------------------------------------------------------------
// 32 bytes at any alignment as four little-endian words
LWE_DEV void load32_le(const uint8_t *p, uint64_t w[4]) {
  if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) {
    const uint64_t *q = reinterpret_cast<const uint64_t *>(p);
#pragma unroll
    for (int i = 0; i < 4; i++) w[i] = q[i];
  } else {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      uint64_t v = 0;
#pragma unroll
      for (int b = 0; b < 8; b++) v |= (uint64_t)p[8 * i + b] << (8 * b);
      w[i] = v;
    }
  }
}

// SHA3-256 of prefix || 32 bytes, built lane by lane (the 33-byte message
// is the 32 bytes shifted up one byte; padding opens byte 1 of lane 4)
LWE_DEV void sha3_prefixed32(uint8_t prefix, const uint8_t *msg32, uint64_t s[25]) {
  uint64_t w[4];
  load32_le(msg32, w);
  s[0] = (uint64_t)prefix | (w[0] << 8);
#pragma unroll
  for (int j = 1; j < 4; j++) s[j] = (w[j - 1] >> 56) | (w[j] << 8);
  s[4] = (w[3] >> 56) | ((uint64_t)0x06 << 8);
#pragma unroll
  for (int j = 5; j < 25; j++) s[j] = 0;
  s[SHA3_RATE / 8 - 1] ^= 0x8000000000000000ull;
  keccak_f1600(s);
}

__global__ void k_keygen_seeds(KeygenSeedArgs a) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.count) return;
  const uint8_t *ms = a.ms + 32 * (size_t)e;
  uint64_t s[25];
  uint8_t *pk = a.pk + (size_t)e * a.pk_bytes;
  uint8_t *sk = a.sk + (size_t)e * a.sk_bytes;
  uint8_t *ws = a.ws_seeds + 32 * (size_t)e;
  sha3_prefixed32(0x41, ms, s);  // seedA
  sha3_digest16(s, pk);
  sha3_digest16(s, sk + a.sk_pk_off);
  sha3_digest16(s, ws);
  sha3_prefixed32(0x53, ms, s);  // seedSE
  sha3_digest16(s, ws + 16);
  {
    const uint32_t key[4] = {(uint32_t)s[0], (uint32_t)(s[0] >> 32), (uint32_t)s[1],
                             (uint32_t)(s[1] >> 32)};
    uint32_t rk[44];
    aes_key_expand_global(g_aes_T0, key, rk);
    uint4 *dst = reinterpret_cast<uint4 *>(a.ws_rk + 44 * (size_t)e);
#pragma unroll
    for (int i = 0; i < 11; i++) dst[i] = make_uint4(rk[4 * i], rk[4 * i + 1], rk[4 * i + 2], rk[4 * i + 3]);
  }
  sha3_prefixed32(0x5A, ms, s);  // z
  sha3_digest(s, sk + a.sk_z_off);
}

// Alg. 4 / 5 seeds of the (re-)encryption.  mu is 8 B bytes (B <= 4), i.e.
// whole 64-bit lanes, so both messages are built lane by lane with
// compile-time state indices (nothing leaves the registers):
//   Encaps: mu = H(0x4D || coins)[0 : 8 B]
//   K' = H(pkh || mu),  seedSE' = H(0x01 || pkh || mu)[0 : 16]
__global__ void k_derive(DeriveArgs a) {
  __shared__ uint32_t sT0[256];  // the key expansion's S-box lookups stay on chip
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) sT0[i] = g_aes_T0[i];
  __syncthreads();
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.count) return;
  uint64_t s[25];
  uint64_t *mu64 = reinterpret_cast<uint64_t *>(a.mu + 32 * (size_t)e);
  const uint32_t nb = a.mu_bytes / 8;  // lanes of mu, 1..4
  uint64_t x[8];                       // pkh (4 lanes) || mu (nb lanes) || zeros
  if (a.coins) {
    sha3_prefixed32(0x4D, a.coins + 32 * (size_t)e, s);
#pragma unroll
    for (int i = 0; i < 4; i++) {
      x[4 + i] = (uint32_t)i < nb ? s[i] : 0;
      mu64[i] = x[4 + i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; i++) x[4 + i] = (uint32_t)i < nb ? mu64[i] : 0;
  }
  const uint8_t *pkh = a.pkh_ptrs ? a.pkh_ptrs[e] + a.pkh_off : a.pkh + (size_t)e * a.pkh_stride;
  load32_le(pkh, x);
  // K' = H(pkh || mu): 32 + 8 nb bytes, padding opens lane 4 + nb
  // (every lane is written unconditionally with a selected value: a
  // conditional store to lane 4 + nb would become a dynamically indexed
  // state, i.e. local memory)
#pragma unroll
  for (int i = 0; i < 25; i++) s[i] = i < 8 ? x[i] : 0;
#pragma unroll
  for (int i = 5; i < 9; i++) s[i] ^= (uint32_t)i == 4 + nb ? 0x06ull : 0ull;
  s[SHA3_RATE / 8 - 1] ^= 0x8000000000000000ull;
  keccak_f1600(s);
  sha3_digest(s, a.kprime + 32 * (size_t)e);
  // seedSE' = H(0x01 || pkh || mu): the same lanes one byte later; the
  // padding byte lands in byte 1 of lane 4 + nb
  s[0] = 0x01 | (x[0] << 8);
#pragma unroll
  for (int j = 1; j < 9; j++) s[j] = (x[j - 1] >> 56) | (j < 8 ? x[j] << 8 : 0);
#pragma unroll
  for (int j = 9; j < 25; j++) s[j] = 0;
#pragma unroll
  for (int i = 5; i < 9; i++) s[i] ^= (uint32_t)i == 4 + nb ? 0x0600ull : 0ull;
  s[SHA3_RATE / 8 - 1] ^= 0x8000000000000000ull;
  keccak_f1600(s);
  sha3_digest16(s, a.seeds + 32 * (size_t)e);
  const uint32_t key[4] = {(uint32_t)s[0], (uint32_t)(s[0] >> 32), (uint32_t)s[1],
                           (uint32_t)(s[1] >> 32)};
  uint32_t rk[44];
  aes_key_expand_global(sT0, key, rk);
  uint4 *dst = reinterpret_cast<uint4 *>(a.rk + 44 * (size_t)e);
#pragma unroll
  for (int i = 0; i < 11; i++) dst[i] = make_uint4(rk[4 * i], rk[4 * i + 1], rk[4 * i + 2], rk[4 * i + 3]);
}

// Tree hash: tpi threads per message compute its 1024-byte-chunk digests
// into shared memory; threads 0..ipc-1 (one per message, so the root phase
// fills whole warps) then hash the digests -- the root -- and, for Encaps,
// derive the key.  A message's digests sit at a stride of 4 m + 1 words so
// the root threads' 64-bit reads fall in different banks.
__global__ void __launch_bounds__(TREE_MAX_THREADS) k_tree(TreeArgs a) {
  extern __shared__ uint64_t sleaf[];  // [ipc][4 m + 1]
  const uint32_t words = 4 * a.m + 1;
  const uint32_t e0 = blockIdx.x * a.ipc;
  {
    const uint32_t li = threadIdx.x / a.tpi, lt = threadIdx.x % a.tpi;
    const uint32_t e = e0 + li;
    if (li < a.ipc && e < a.count) {
      const uint8_t *msg = a.msg_ptrs ? a.msg_ptrs[e] : a.msgs + (size_t)e * a.stride;
      uint64_t *mine = sleaf + (size_t)li * words;
      uint64_t s[25];
      for (uint32_t c = lt; c < a.m; c += a.tpi) {
        const uint32_t off = c * LWE_TREE_CHUNK;
        sha3_256_global(msg + off, min((uint32_t)LWE_TREE_CHUNK, a.len - off), s);
        mine[4 * c] = s[0];
        mine[4 * c + 1] = s[1];
        mine[4 * c + 2] = s[2];
        mine[4 * c + 3] = s[3];
      }
    }
  }
  __syncthreads();
  const uint32_t e = e0 + threadIdx.x;
  if (threadIdx.x >= a.ipc || e >= a.count) return;
  uint64_t s[25];
  sha3_256_mem(reinterpret_cast<const uint8_t *>(sleaf + (size_t)threadIdx.x * words), 32 * a.m, s);
  if (a.mode == TREE_DIGEST) {
    sha3_digest(s, a.out + (size_t)e * a.out_stride);
    if (a.out2) sha3_digest(s, a.out2 + (size_t)e * a.out2_stride);
    return;
  }
  // Encaps (Alg. 4): K = H(K' || H(c))
  uint64_t lanes[SHA3_RATE / 8];
  lanes_zero(lanes);
  const uint64_t *kp = reinterpret_cast<const uint64_t *>(a.kprime + 32 * (size_t)e);
  for (int i = 0; i < 4; i++) lanes[i] = kp[i];
  for (int i = 0; i < 4; i++) lanes[4 + i] = s[i];
  sha3_256_lanes(lanes, 64, s);
  sha3_digest(s, a.out + 32 * (size_t)e);
}

__global__ void __launch_bounds__(128) k_final_key(FinalKeyArgs a) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.count) return;
  // all-ones when the re-encryption matched (flag == 0), else zero
  const uint32_t f = a.flags[e];
  const uint64_t keep = (uint64_t)0 - (uint64_t)(((f | (0u - f)) >> 31) ^ 1u);
  const uint64_t *kp = reinterpret_cast<const uint64_t *>(a.kprime + 32 * (size_t)e);
  const uint64_t *z = reinterpret_cast<const uint64_t *>(a.z_ptrs ? a.z_ptrs[e] + a.z_off : a.z);
  const uint64_t *hc = reinterpret_cast<const uint64_t *>(a.hc + 32 * (size_t)e);
  uint64_t lanes[SHA3_RATE / 8];
  lanes_zero(lanes);
  for (int i = 0; i < 4; i++) lanes[i] = (kp[i] & keep) | (z[i] & ~keep);
  for (int i = 0; i < 4; i++) lanes[4 + i] = hc[i];
  uint64_t s[25];
  sha3_256_lanes(lanes, 64, s);
  sha3_digest(s, a.K + 32 * (size_t)e);
}

// ---------------------------------------------------------------------------
// Operand preparation of the tensor path: the columns of [A | B] split into
// signed 8-bit limbs, x = lo + 256 hi (mod 2^16), written K-major as bf16
// (limbs[l][c][i]); a 64 x 64 tile is transposed through shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_limbs(GemmLimbArgs a) {
  extern __shared__ uint32_t sT[];
  __shared__ __align__(16) uint16_t tile[64][72];
  const bool fused = (a.A == nullptr);
  const uint32_t n = a.n, ncols = n + (a.B ? 8u : 0u);
  const uint32_t i0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const uint32_t mq = (1u << a.logq) - 1u, mm = mq | (mq << 16);
  AesTab tab;
  uint32_t rk[44];
  if (fused) {
    aes_fill_smem(sT, g_aes_T0);
    __syncthreads();
    tab = aes_tab(sT);
    uint32_t key[4];
    aes_load_key(a.seedA, key);
    aes_key_expand(tab, key, rk);
  }
  for (uint32_t idx = threadIdx.x; idx < 512; idx += blockDim.x) {
    const uint32_t r = idx >> 3, cq = idx & 7;
    const uint32_t i = i0 + r, c = c0 + 8 * cq;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (i < n) {
      if (c + 8 <= n) {
        if (fused) {
          v = aes_ctr_block(tab, rk, 0, (uint64_t)i * (n / 8) + c / 8);
          v.x &= mm;
          v.y &= mm;
          v.z &= mm;
          v.w &= mm;
        } else {
          v = ld_nc_u4(a.A + (size_t)i * n + c);
        }
      } else if (a.B && c == n) {
        v = ld_nc_u4(a.B + 16 * (size_t)i);
      }
    }
    *reinterpret_cast<uint4 *>(&tile[r][8 * cq]) = v;
  }
  __syncthreads();
  for (uint32_t idx = threadIdx.x; idx < 512; idx += blockDim.x) {
    const uint32_t cl = idx >> 3, ic = idx & 7;
    const uint32_t c = c0 + cl, i = i0 + 8 * ic;
    if (c >= ncols || i >= n) continue;
    uint32_t lo[4], hi[4];
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      float fl[2], fh[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int x = tile[8 * ic + t + u][cl];
        const int l = (int)(int8_t)(uint8_t)(x & 0xff);
        const int h = (int)(int8_t)(uint8_t)(((x - l) >> 8) & 0xff);
        fl[u] = (float)l;
        fh[u] = (float)h;
      }
      __nv_bfloat162 bl = __floats2bfloat162_rn(fl[0], fl[1]);
      __nv_bfloat162 bh = __floats2bfloat162_rn(fh[0], fh[1]);
      lo[t / 2] = *reinterpret_cast<uint32_t *>(&bl);
      hi[t / 2] = *reinterpret_cast<uint32_t *>(&bh);
    }
    uint16_t *L = a.limbs;
    *reinterpret_cast<uint4 *>(L + (size_t)c * n + i) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4 *>(L + ((size_t)ncols + c) * n + i) =
        make_uint4(hi[0], hi[1], hi[2], hi[3]);
  }
}

__global__ void k_s_to_bf16(const int8_t *__restrict__ S, uint64_t count, uint16_t *out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    __nv_bfloat16 b = __float2bfloat16_rn((float)S[i]);
    out[i] = *reinterpret_cast<uint16_t *>(&b);
  }
}

// ---------------------------------------------------------------------------
// Host-side launch wrappers (called from lwe_api.cu)
// ---------------------------------------------------------------------------
static int grid_for(uint64_t work, int per_cta, int max_ctas) {
  uint64_t g = (work + per_cta - 1) / per_cta;
  if (g > (uint64_t)max_ctas) g = max_ctas;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t lwe_upload_aes_table(const uint32_t T0[256]) {
  return cudaMemcpyToSymbol(g_aes_T0, T0, 256 * sizeof(uint32_t));
}

cudaError_t lwe_kernel_smem_setup() {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_expand_A, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_noise, cudaFuncAttributeMaxDynamicSharedMemorySize, NOISE_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_mul_as<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int fused_smem = AES_SMEM_BYTES + SA_CH * 32;
  e = cudaFuncSetAttribute(k_mul_sa_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fused_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_mul_sa_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fused_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_limbs, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  return e;
}

void launch_expand_A(const uint8_t *seeds, uint32_t seed_stride, uint32_t count, uint32_t n,
                     uint32_t logq, uint16_t *A, uint64_t a_stride, int num_sms, cudaStream_t st) {
  const uint64_t nblk = (uint64_t)n * n / 8;
  const int gx = grid_for(nblk, 512 * 4, num_sms);
  k_expand_A<<<dim3(gx, count), 512, AES_SMEM_BYTES, st>>>(seeds, seed_stride, n, logq, A, a_stride);
}

void launch_noise(const NoiseArgs &a, int num_sms, cudaStream_t st) {
  const int g = grid_for((uint64_t)a.count * a.runs_per_item, 16, num_sms);
  k_noise<<<g, 512, NOISE_SMEM_BYTES, st>>>(a);
}

void launch_mul_as(const MulAsArgs &a, uint32_t count, bool fused, cudaStream_t st) {
  dim3 grid((a.n + 7) / 8, count);
  if (fused)
    k_mul_as<true><<<grid, 256, AES_SMEM_BYTES, st>>>(a);
  else
    k_mul_as<false><<<grid, 256, 0, st>>>(a);
}

void launch_decrypt(const DecryptArgs &a, uint32_t count, cudaStream_t st) {
  k_decrypt<<<count, 256, 0, st>>>(a);
}

void launch_mul_sa(const MulSaArgs &a, uint32_t items, bool fused, bool cmp, cudaStream_t st) {
  dim3 grid((a.n + 63) / 64, items);
  if (fused) {
    const int smem = AES_SMEM_BYTES + SA_CH * 32;
    if (cmp)
      k_mul_sa_fused<true><<<grid, 256, smem, st>>>(a);
    else
      k_mul_sa_fused<false><<<grid, 256, smem, st>>>(a);
  } else {
    if (cmp)
      k_mul_sa<true><<<grid, 256, 0, st>>>(a);
    else
      k_mul_sa<false><<<grid, 256, 0, st>>>(a);
  }
}

void launch_v_encode(const VEncArgs &a, uint32_t count, bool cmp, cudaStream_t st) {
  if (cmp)
    k_v_encode<true><<<count, 256, 0, st>>>(a);
  else
    k_v_encode<false><<<count, 256, 0, st>>>(a);
}

void launch_keygen_seeds(const KeygenSeedArgs &a, cudaStream_t st) {
  k_keygen_seeds<<<(a.count + 63) / 64, 64, 0, st>>>(a);
}

void launch_derive(const DeriveArgs &a, cudaStream_t st) {
  k_derive<<<(a.count + 63) / 64, 64, 0, st>>>(a);
}

// One CTA per SM where the batch allows (the leaf work is one wave: CTAs of
// equal size spread it evenly), at most TREE_MAX_THREADS threads and 48 KB
// of digests per CTA.
void launch_tree(TreeArgs &a, int num_sms, cudaStream_t st) {
  a.m = (a.len + LWE_TREE_CHUNK - 1) / LWE_TREE_CHUNK;
  uint32_t t = 1;
  while (t < a.m && t < 256) t <<= 1;
  a.tpi = t;
  const uint32_t words = 4 * a.m + 1;
  uint32_t cap = TREE_MAX_THREADS / t;
  cap = std::min<uint32_t>(cap, (48u * 1024u) / (8u * words));
  cap = std::max<uint32_t>(cap, 1u);
  const uint32_t sms = num_sms > 0 ? (uint32_t)num_sms : 1u;
  a.ipc = std::min<uint32_t>(cap, (a.count + sms - 1) / sms);
  if (a.ipc == 0) a.ipc = 1;
  const uint32_t threads = (a.ipc * t + 31) / 32 * 32;
  const size_t smem = (size_t)a.ipc * words * 8;
  k_tree<<<(a.count + a.ipc - 1) / a.ipc, threads, smem, st>>>(a);
}

void launch_final_key(const FinalKeyArgs &a, cudaStream_t st) {
  k_final_key<<<(a.count + 127) / 128, 128, 0, st>>>(a);
}

void launch_gemm_limbs(const GemmLimbArgs &a, int num_sms, cudaStream_t st) {
  (void)num_sms;
  const uint32_t ncols = a.n + (a.B ? 8u : 0u);
  dim3 grid((ncols + 63) / 64, (a.n + 63) / 64);
  k_limbs<<<grid, 256, a.A ? 0 : AES_SMEM_BYTES, st>>>(a);
}

void launch_s_to_bf16(const int8_t *S, uint64_t count, uint16_t *out, int num_sms, cudaStream_t st) {
  const int g = grid_for(count, 256 * 8, num_sms * 8);
  k_s_to_bf16<<<g, 256, 0, st>>>(S, count, out);
}
