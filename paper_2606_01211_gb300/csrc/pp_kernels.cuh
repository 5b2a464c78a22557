// pp_kernels.cuh -- the paper's own parameter profile (Tab. 1): odd q in
// {3329, 12289, 65537}, a 256-bit message encrypted bit by bit (Alg. 2 run
// for 256 columns r_k at once), a binomial secret (eta = 3), Gaussian e, r,
// e1 and a centred-uniform e2, threshold decoding (Alg. 3).  Entries mod q
// are uint32; products accumulate in int32 with A centred to (-q/2, q/2]
// and a reduction mod q at least every 4096 terms, so no sum exceeds 2^31.
//
// Included once, by kem_kernels.cu (it uses that file's AES table).
#pragma once
#include "pp_types.h"

#define PP_A_DOMAIN 16  // stream domain of A's first try; try t uses 16 + t
#define PP_A_TRIES 8
#define PP_REDUCE_EVERY 4096

// x mod q for x < 2^32 by Barrett reduction: m = floor(2^32 / q), so the
// estimated quotient is low by at most one
LWE_DEV uint32_t mod_u32(uint32_t x, ModQ M) {
  const uint32_t r = x - __umulhi(x, M.m) * M.q;
  return r >= M.q ? r - M.q : r;
}

LWE_DEV uint32_t mod_s32(int32_t x, ModQ M) {  // |x| < 2^31
  const uint32_t r = mod_u32((uint32_t)(x < 0 ? -x : x), M);
  return (x < 0 && r) ? M.q - r : r;
}

LWE_DEV int32_t centre(uint32_t a, uint32_t q) {
  return a > q / 2 ? (int32_t)a - (int32_t)q : (int32_t)a;
}

// ---------------------------------------------------------------------------
// A (Alg. 1) uniform mod q by rejection: entry (i, j) is 32-bit word
// i n + j of the stream (seedA, domain 16 + t), accepted when below the
// largest multiple of q under 2^32; a rejected word moves to the next try.
// A counter block holds 4 consecutive entries of a row; a warp takes runs
// of 128 blocks (4 per lane, two at a time) inside one 256-aligned counter
// window of the first try's stream (aes_ctr_run).
// ---------------------------------------------------------------------------
// Entries of blocks ba (w[0..3]) and bb (w[4..7]): the rare rejected words
// are replaced from the next tries (one AES block each), then all reduced
// mod q; an entry rejected by every try is 0.
LWE_DEV void pp_a_accept(const AesTab &tab, const uint32_t rk[44], uint64_t ba, uint64_t bb,
                         uint32_t limit, ModQ M, uint32_t w[8]) {
  uint32_t bad = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) bad |= (w[c] >= limit ? 1u : 0u) << c;
  uint32_t zero = 0;
  while (bad) {  // probability < q / 2^32 per entry
    const int c = __ffs(bad) - 1;
    bad &= bad - 1;
    bool ok = false;
    for (uint32_t t = 1; !ok && t < PP_A_TRIES; t++) {
      const uint4 u = aes_ctr_block(tab, rk, PP_A_DOMAIN + t, c < 4 ? ba : bb);
      const uint32_t x = (c & 3) == 0 ? u.x : (c & 3) == 1 ? u.y : (c & 3) == 2 ? u.z : u.w;
      if (x < limit) {
#pragma unroll
        for (int d = 0; d < 8; d++)
          if (d == c) w[d] = x;
        ok = true;
      }
    }
    if (!ok) zero |= 1u << c;
  }
#pragma unroll
  for (int c = 0; c < 8; c++) w[c] = (zero >> c) & 1u ? 0u : mod_u32(w[c], M);
}

__global__ void __launch_bounds__(512, 1) k_pp_expand_A(const uint8_t *__restrict__ seedA,
                                                     uint32_t n, ModQ M, uint32_t *__restrict__ A) {
  extern __shared__ uint32_t sT[];
  pdl_trigger();
  aes_fill_smem(sT, g_aes_img);
  __syncthreads();
  pdl_wait();
  const AesTab tab = aes_tab(sT);
  uint32_t key[4], rk[44];
  aes_load_key(seedA, key);
  aes_key_expand(tab, key, rk);
  const uint32_t limit = (uint32_t)((0x100000000ull / M.q) * M.q);
  const uint64_t nblk = (uint64_t)n * n / 4;
  uint4 *out = reinterpret_cast<uint4 *>(A);
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nruns = (nblk + 127) / 128, nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t run = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); run < nruns;
       run += nw) {
    const uint64_t first = run * 128;
    const AesCtrRun win = aes_ctr_run(tab, rk, PP_A_DOMAIN, first);
    const uint32_t x0 = (uint32_t)(first & 255u) + lane;
#pragma unroll 1
    for (uint32_t j = 0; j < 4; j += 2) {
      const uint64_t ba = first + lane + 32 * j, bb = ba + 32;
      if (ba >= nblk) break;
      const uint4 va = aes_ctr_run_block(tab, rk, win, x0 + 32 * j);
      const uint4 vb = bb < nblk ? aes_ctr_run_block(tab, rk, win, x0 + 32 * j + 32)
                                 : make_uint4(0, 0, 0, 0);
      uint32_t w[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
      pp_a_accept(tab, rk, ba, bb, limit, M, w);
      out[ba] = make_uint4(w[0], w[1], w[2], w[3]);
      if (bb < nblk) out[bb] = make_uint4(w[4], w[5], w[6], w[7]);
    }
  }
}

// ---------------------------------------------------------------------------
// Noise streams (key schedule rk, one item): binomial eta = 3 from one byte
// per sample, the CDF-table Gaussian from one 16-bit word, or the centred
// uniform floor((2k + 1) w / 2^16) - k from one 16-bit word.
// ---------------------------------------------------------------------------
LWE_DEV uint32_t pp_noise_blocks(const PpNoiseOut &o) {
  return o.kind == PP_BINOMIAL ? (o.count + 15) / 16 : (o.count + 7) / 8;
}

__global__ void __launch_bounds__(512, 1) k_pp_noise(PpNoiseArgs a) {
  extern __shared__ uint32_t sT[];
  pdl_trigger();
  aes_fill_smem(sT, g_aes_img);
  __syncthreads();
  pdl_wait();
  const AesTab tab = aes_tab(sT);
  uint32_t rk[44];
#pragma unroll
  for (int i = 0; i < 44; i++) rk[i] = a.rk[i];
  uint32_t nb[3] = {0, 0, 0};
  uint64_t total = 0;
  for (uint32_t s = 0; s < a.nout; s++) {
    nb[s] = pp_noise_blocks(a.o[s]);
    total += nb[s];
  }
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s = 0;
    uint64_t b = g;
    while (s + 1 < a.nout && b >= nb[s]) {
      b -= nb[s];
      s++;
    }
    const PpNoiseOut o = a.o[s];
    const uint4 v = aes_ctr_block(tab, rk, o.domain, b);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    if (o.kind == PP_BINOMIAL) {
      int8_t *dst = reinterpret_cast<int8_t *>(o.out);
#pragma unroll
      for (int t = 0; t < 16; t++) {
        const uint32_t x = (w[t >> 2] >> (8 * (t & 3))) & 0xffu;
        const int e = __popc(x & 7u) - __popc((x >> 3) & 7u);
        const uint64_t idx = 16 * b + t;
        if (idx < o.count) dst[idx] = (int8_t)e;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 8; t++) {
        const uint32_t h = (w[t >> 1] >> (16 * (t & 1))) & 0xffffu;
        int e;
        if (o.kind == PP_GAUSS) {
          const uint32_t tt = h >> 1;
          int mag = 0;
          for (uint32_t i = 0; i < a.clip; i++) mag += tt > a.T[i] ? 1 : 0;
          e = (h & 1u) ? -mag : mag;
        } else {
          e = (int)(((2u * a.kunif + 1u) * h) >> 16) - (int)a.kunif;
        }
        const uint64_t idx = 8 * b + t;
        if (idx < o.count) {
          if (o.kind == PP_GAUSS)
            reinterpret_cast<int8_t *>(o.out)[idx] = (int8_t)e;
          else
            reinterpret_cast<int32_t *>(o.out)[idx] = e;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// KeyGen (Alg. 1): t = A s + e mod q, warp per row, written to the
// public key and to the copy of it inside the secret key.
// ---------------------------------------------------------------------------
LWE_DEV uint32_t warp_sum_mod(uint32_t x, ModQ M) {  // x < q on every lane
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return mod_u32(x, M);  // < 32 q < 2^32
}

__global__ void __launch_bounds__(256) k_pp_as(PpAsArgs a) {
  pdl_trigger();
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= a.n) return;
  const uint32_t *row = a.A + (size_t)i * a.n;
  int32_t acc = 0;
  uint32_t red = 0, since = 0;
  for (uint32_t j = 4 * lane; j < a.n; j += 128) {
    const uint4 x = ld_nc_u4(row + j);
    const char4 s = *reinterpret_cast<const char4 *>(a.s + j);
    acc += centre(x.x, a.M.q) * s.x + centre(x.y, a.M.q) * s.y + centre(x.z, a.M.q) * s.z +
           centre(x.w, a.M.q) * s.w;
    if ((since += 4) >= PP_REDUCE_EVERY) {
      red = mod_u32(red + mod_s32(acc, a.M), a.M);
      acc = 0;
      since = 0;
    }
  }
  red = mod_u32(red + mod_s32(acc, a.M), a.M);
  const uint32_t sum = warp_sum_mod(red, a.M);
  if (lane == 0) {
    const uint32_t t = mod_u32(sum + mod_s32(a.e[i], a.M), a.M);
    a.t[i] = t;
    if (a.t2) a.t2[i] = t;
  }
}

// ---------------------------------------------------------------------------
// Encrypt's products (Alg. 2 for the 256 columns r_k at once):
// U^T = R^T A + E1^T (mod q), R^T 256 x n int8, A n x n, as a CUDA-core GEMM.
// CTA = 64 rows k x 64 columns j; thread (ty, tx) holds 4 x 4 sums; A tiles
// of 32 x 64 (centred, int32) and R^T tiles of 64 x 32 (transposed to
// [i][k], so 4 rows k are one 32-bit word) are staged in shared memory.
// CMP (Decaps' re-encryption): compare with the received U^T instead of
// storing, and flag a mismatch.
// ---------------------------------------------------------------------------

#define PPE_BM 64
#define PPE_BN 64
#define PPE_BK 32

template <bool CMP>
__global__ void __launch_bounds__(256) k_pp_encrypt(PpEncArgs a) {
  __shared__ __align__(16) int32_t As[PPE_BK][PPE_BN];
  __shared__ __align__(16) int8_t Rs[PPE_BK][PPE_BM];
  pdl_trigger();
  pdl_wait();
  const uint32_t n = a.n, q = a.M.q;
  const uint32_t j0 = blockIdx.x * PPE_BN, k0 = blockIdx.y * PPE_BM;
  const uint32_t tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int32_t acc[4][4];
  uint32_t red[4][4];
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) acc[r][c] = 0, red[r][c] = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += PPE_BK) {
    // A tile: 32 rows x 64 columns = 512 uint4, two per thread
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const uint32_t idx = tid + 256 * u, row = idx >> 4, c4 = idx & 15;
      const uint4 x = ld_nc_u4(a.A + (size_t)(i0 + row) * n + j0 + 4 * c4);
      *reinterpret_cast<int4 *>(&As[row][4 * c4]) =
          make_int4(centre(x.x, q), centre(x.y, q), centre(x.z, q), centre(x.w, q));
    }
    // R^T tile: 64 rows k x 32 columns i = 2048 bytes, 8 per thread
    {
      const uint32_t kk = tid >> 2, i8 = 8 * (tid & 3);
      const uint2 r = ld_nc_u2(a.Rt + (size_t)(k0 + kk) * n + i0 + i8);
#pragma unroll
      for (int b = 0; b < 8; b++)
        Rs[i8 + b][kk] = (int8_t)((b < 4 ? r.x >> (8 * b) : r.y >> (8 * (b - 4))) & 0xff);
    }
    __syncthreads();
#pragma unroll 8
    for (int ii = 0; ii < PPE_BK; ii++) {
      const int4 x = *reinterpret_cast<const int4 *>(&As[ii][4 * tx]);
      const uint32_t rw = *reinterpret_cast<const uint32_t *>(&Rs[ii][4 * ty]);
      const int xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const int rv = (int)(int8_t)(rw >> (8 * r));
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] += rv * xv[c];
      }
    }
    __syncthreads();
    if ((i0 + PPE_BK) % PP_REDUCE_EVERY == 0) {
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          red[r][c] = mod_u32(red[r][c] + mod_s32(acc[r][c], a.M), a.M);
          acc[r][c] = 0;
        }
    }
  }
  uint32_t diff = 0;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const uint32_t k = k0 + 4 * ty + r, j = j0 + 4 * tx;
    const char4 e = *reinterpret_cast<const char4 *>(a.E1t + (size_t)k * n + j);
    const int ev[4] = {e.x, e.y, e.z, e.w};
    uint32_t val[4];
#pragma unroll
    for (int c = 0; c < 4; c++)
      val[c] = mod_u32(mod_u32(red[r][c] + mod_s32(acc[r][c], a.M), a.M) + mod_s32(ev[c], a.M),
                       a.M);
    uint4 *o = reinterpret_cast<uint4 *>(a.Ut + (size_t)k * n + j);
    if (CMP) {
      const uint4 g = *o;
      diff |= (g.x ^ val[0]) | (g.y ^ val[1]) | (g.z ^ val[2]) | (g.w ^ val[3]);
    } else {
      *o = make_uint4(val[0], val[1], val[2], val[3]);
    }
  }
  if (CMP) {
    diff = __reduce_or_sync(0xffffffffu, diff);
    if ((tid & 31) == 0 && diff) atomicOr(a.flags, 1u);
  }
}

// ---------------------------------------------------------------------------
// v_k = t^T r_k + e2_k + m_k floor(q/2) (mod q) (Alg. 2), CTA per k;
// CMP compares with the received v.
// ---------------------------------------------------------------------------

// sum_i centre(x_i) s_i (mod q) over i < n (n a multiple of 4) by a whole
// CTA of 8 warps: a lane takes 4 consecutive entries, the warps interleave
// in steps of 1024 entries, and the 8 warp sums meet in shared memory.  One
// message bit per CTA keeps every SM busy where one warp per bit (256
// warps in 32 CTAs) walked n / 128 dependent loads in a row.
LWE_DEV uint32_t pp_cta_dot_mod(const uint32_t *x, const int8_t *s, uint32_t n, ModQ M) {
  __shared__ uint32_t part[8];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t acc = 0;
  uint32_t red = 0, since = 0;
  for (uint32_t i = 4 * (lane + 32 * w); i < n; i += 1024) {
    const uint4 v = ld_nc_u4(x + i);
    const char4 c = *reinterpret_cast<const char4 *>(s + i);
    acc += centre(v.x, M.q) * c.x + centre(v.y, M.q) * c.y + centre(v.z, M.q) * c.z +
           centre(v.w, M.q) * c.w;
    if ((since += 4) >= PP_REDUCE_EVERY) {
      red = mod_u32(red + mod_s32(acc, M), M);
      acc = 0;
      since = 0;
    }
  }
  red = mod_u32(red + mod_s32(acc, M), M);
  const uint32_t ws = warp_sum_mod(red, M);
  if (lane == 0) part[w] = ws;
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) tot = mod_u32(tot + part[j], M);
  return tot;
}

template <bool CMP>
__global__ void __launch_bounds__(256) k_pp_v(PpVArgs a) {
  pdl_trigger();
  pdl_wait();
  const uint32_t k = blockIdx.x;  // message bit
  const uint32_t sum = pp_cta_dot_mod(a.t, a.Rt + (size_t)k * a.n, a.n, a.M);
  if (threadIdx.x == 0) {
    const uint32_t bit = (a.m[k >> 3] >> (k & 7)) & 1u;
    const uint32_t v = mod_u32(mod_u32(sum + mod_s32(a.e2[k], a.M), a.M) + bit * (a.M.q / 2), a.M);
    if (CMP) {
      if (a.v[k] != v) atomicOr(a.flags, 1u);
    } else {
      a.v[k] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Decrypt (Alg. 3): mu_k = v_k - s^T u_k (mod q), CTA per k; bit k of m is
// 1 iff q < 4 mu_k < 3q.  m (8 words, zeroed by the caller) gathers the bits.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_pp_decrypt(PpDecArgs a) {
  pdl_trigger();
  pdl_wait();
  const uint32_t k = blockIdx.x;  // message bit
  const uint32_t su = pp_cta_dot_mod(a.Ut + (size_t)k * a.n, a.s, a.n, a.M);
  if (threadIdx.x == 0) {
    const uint32_t q = a.M.q, mu = mod_u32(a.v[k] + q - su, a.M);
    const uint64_t m4 = 4ull * mu;
    const uint32_t bit = (m4 > q && m4 < 3ull * q) ? 1u : 0u;
    if (bit) atomicOr(a.m + (k >> 5), 1u << (k & 31));
  }
}

// ---------------------------------------------------------------------------
// The tensor-core form of Encrypt's product: the columns of A split into
// two limbs of its centred value, x = lo + 256 hi with lo in [-128, 127]
// and hi in [-128, 128], written as bf16 K-major (limbs[l][c][i]) for the
// odd-modulus GEMM.  A 64 x 64 tile is transposed through shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_pp_limbs(const uint32_t *__restrict__ A, uint32_t n,
                                                  uint32_t q, uint16_t *__restrict__ L) {
  __shared__ int32_t tile[64][65];
  pdl_trigger();
  pdl_wait();
  const uint32_t i0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  for (uint32_t idx = threadIdx.x; idx < 64 * 16; idx += blockDim.x) {
    const uint32_t r = idx >> 4, c4 = idx & 15;
    const uint4 x = ld_nc_u4(A + (size_t)(i0 + r) * n + c0 + 4 * c4);
    tile[r][4 * c4] = centre(x.x, q);
    tile[r][4 * c4 + 1] = centre(x.y, q);
    tile[r][4 * c4 + 2] = centre(x.z, q);
    tile[r][4 * c4 + 3] = centre(x.w, q);
  }
  __syncthreads();
  for (uint32_t idx = threadIdx.x; idx < 64 * 8; idx += blockDim.x) {
    const uint32_t cl = idx >> 3, ic = idx & 7;
    uint32_t lo[4], hi[4];
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      float fl[2], fh[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int x = tile[8 * ic + t + u][cl];
        const int l = (int)(int8_t)(uint8_t)(x & 0xff);
        fl[u] = (float)l;
        fh[u] = (float)((x - l) >> 8);
      }
      __nv_bfloat162 bl = __floats2bfloat162_rn(fl[0], fl[1]);
      __nv_bfloat162 bh = __floats2bfloat162_rn(fh[0], fh[1]);
      lo[t / 2] = *reinterpret_cast<uint32_t *>(&bl);
      hi[t / 2] = *reinterpret_cast<uint32_t *>(&bh);
    }
    const size_t at = (size_t)(c0 + cl) * n + i0 + 8 * ic;
    *reinterpret_cast<uint4 *>(L + at) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4 *>(L + (size_t)n * n + at) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  }
}
