// kem_kernels.cu -- CUDA-core kernels of the plain-LWE KEM hot path (sm_103a).
//
//   k_expand_A      sample(seedA) of Alg. 1: AES-128-CTR expansion of A,
//                   16-byte coalesced stores.
//   k_noise         the error/secret distributions of Alg. 1-2 (Tab. 1:
//                   rounded Gaussian) by CDF-table inverse sampling of AES
//                   counter streams.
//   k_mul_as_rows, k_mul_as_fused: B = A S + E of Alg. 1 (A stored, or
//                   regenerated from its seed in-CTA).
//   k_decrypt       M = C - B' S and mu' = Dec(M) of Alg. 3.
//   k_sa            B' = S' A + E' of Alg. 2 on the CUDA cores (A stored or
//                   regenerated from its seed in-CTA), with a compare
//                   epilogue for Alg. 5.
//   k_v_encode      V = S' B + E'', C = V + Enc(mu) of Alg. 2 (or compare).
//   k_keygen_seeds, k_derive, k_tree, k_final_key: the hashing of
//                   Alg. 4-5 (SHA3-256) and the Fujisaki-Okamoto selection.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "aes.cuh"
#include "common.cuh"
#include "gemm_tc.h"
#include "kem_kernels.h"
#include "pp_types.h"
#include "keccak_warp.cuh"

// The round table T0 (see aes.cuh) and the replicated shared-memory image of
// all four tables; both written by lwe_upload_aes_table.
__device__ uint32_t g_aes_T0[256];
__device__ uint4 g_aes_img[AES_TABLE_WORDS / 4];

// ---------------------------------------------------------------------------
// A expansion: a warp per run of 128 counter blocks (16-byte blocks of A),
// grid-stride over the runs; one key per grid.y.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512, 1) k_expand_A(const uint8_t *__restrict__ seeds,
                                                  uint32_t seed_stride, uint32_t n,
                                                  uint32_t logq, uint16_t *__restrict__ A,
                                                  uint64_t a_stride) {
  extern __shared__ uint32_t sT[];
  pdl_trigger();
  aes_fill_smem(sT, g_aes_img);
  __syncthreads();
  pdl_wait();
  const AesTab tab = aes_tab(sT);
  const uint32_t e = blockIdx.y;
  uint32_t key[4], rk[44];
  aes_load_key(seeds + (size_t)e * seed_stride, key);
  aes_key_expand(tab, key, rk);
  const uint32_t m = (1u << logq) - 1u;
  const uint32_t mm = m | (m << 16);
  const uint64_t nblk = (uint64_t)n * n / 8;
  uint4 *out = reinterpret_cast<uint4 *>(A + (size_t)e * a_stride);
  // a warp takes runs of 128 consecutive blocks (4 per lane, two at a time);
  // a run lies inside one 256-aligned counter window (aes_ctr_run), whose
  // constants are worked out for 32 runs at a time, one per lane, and
  // passed to the warp by shuffles as in noise_runs
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nruns = (nblk + 127) / 128, nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (uint64_t g = 0; gw + nw * g < nruns; g += 32) {
    AesCtrRun mine{};
    if (gw + nw * (g + lane) < nruns) mine = aes_ctr_run(tab, rk, 0, (gw + nw * (g + lane)) * 128);
    for (uint32_t jr = 0; jr < 32; jr++) {
      const uint64_t run = gw + nw * (g + jr);
      if (run >= nruns) break;  // the same for every lane
      const uint64_t first = run * 128;
      const AesCtrRun win = aes_ctr_run_shfl(mine, jr);
      const uint32_t x0 = (uint32_t)(first & 255u) + lane;
      if (first + 128 <= nblk) {
#pragma unroll
        for (uint32_t j = 0; j < 4; j += 2) {
          uint4 va = aes_ctr_run_block(tab, rk, win, x0 + 32 * j);
          uint4 vb = aes_ctr_run_block(tab, rk, win, x0 + 32 * j + 32);
          out[first + lane + 32 * j] = make_uint4(va.x & mm, va.y & mm, va.z & mm, va.w & mm);
          out[first + lane + 32 * j + 32] = make_uint4(vb.x & mm, vb.y & mm, vb.z & mm, vb.w & mm);
        }
      } else {
#pragma unroll 1
        for (uint32_t x = x0; first + (x - x0) + lane < nblk; x += 32) {
          const uint4 v = aes_ctr_run_block(tab, rk, win, x);
          out[first + (x - x0) + lane] = make_uint4(v.x & mm, v.y & mm, v.z & mm, v.w & mm);
        }
      }
    }
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

// The runs of one warp: warp `gwarp` of `nwarps` takes runs gwarp,
// gwarp + nwarps, ...  A run's window constants (aes_ctr_run: 27 lookups)
// are the same for all 32 lanes, so they are worked out for 32 runs at a
// time, lane l for the warp's (g + l)-th run with that run's item key, and
// passed to the whole warp by shuffles when the run comes up: 27 lookup
// instructions per 32 runs instead of per run.
struct NoiseRun {
  uint32_t e, r, s;  // item, run within the item's streams, stream
};

LWE_DEV NoiseRun noise_run_of(const NoiseArgs &a, uint64_t run) {
  NoiseRun x;
  x.e = (uint32_t)(run / a.runs_per_item);
  x.r = (uint32_t)(run % a.runs_per_item);
  x.s = 0;
  while (x.s + 1 < a.nout && x.r >= a.out[x.s].runs) {
    x.r -= a.out[x.s].runs;
    x.s++;
  }
  return x;
}

LWE_DEV void noise_load_rk(const NoiseArgs &a, uint32_t e, uint32_t rk[44]) {
  const uint4 *rkp = reinterpret_cast<const uint4 *>(a.rk + 44 * (size_t)e);
#pragma unroll
  for (int i = 0; i < 11; i++) {
    const uint4 v = __ldg(rkp + i);
    rk[4 * i] = v.x;
    rk[4 * i + 1] = v.y;
    rk[4 * i + 2] = v.z;
    rk[4 * i + 3] = v.w;
  }
}

LWE_DEV void noise_runs(const NoiseArgs &a, const AesTab &tab, const char *smem, uint64_t gwarp,
                        uint64_t nwarps) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nruns = (uint64_t)a.count * a.runs_per_item;
  for (uint64_t g = 0; gwarp + nwarps * g < nruns; g += 32) {
    // window constants of this warp's runs g .. g + 31, one per lane
    AesCtrRun mine{};
    {
      const uint64_t run = gwarp + nwarps * (g + lane);
      if (run < nruns) {
        const NoiseRun x = noise_run_of(a, run);
        if (LWE_BOUNDS(x.e < a.count, 108)) {
          uint32_t rk[44];
          noise_load_rk(a, x.e, rk);
          mine = aes_ctr_run(tab, rk, a.out[x.s].domain, x.r * NOISE_RUN);
        }
      }
    }
    for (uint32_t j = 0; j < 32; j++) {
      const uint64_t run = gwarp + nwarps * (g + j);
      if (run >= nruns) break;  // the same for every lane
      const AesCtrRun win = aes_ctr_run_shfl(mine, j);
      const NoiseRun x = noise_run_of(a, run);
      if (!LWE_BOUNDS(x.e < a.count, 108)) continue;
      const NoiseOut o = a.out[x.s];
      uint32_t rk[44];
      noise_load_rk(a, x.e, rk);
      const uint32_t nblk = (o.nsamples + 7) / 8;
      uint8_t *base = reinterpret_cast<uint8_t *>(o.base) + (size_t)x.e * o.item_stride;
      // a run lies inside one 256-aligned window of counter indices, whose
      // first two AES rounds are in `win`
      const uint32_t first = x.r * NOISE_RUN, b0 = first + lane, x0 = (first & 255u) + lane;
      if (first + NOISE_RUN <= nblk) {
        // full run: two independent blocks in flight per lane
#pragma unroll
        for (uint32_t jj = 0; jj < NOISE_RUN / 32; jj += 2) {
          const uint4 va = aes_ctr_run_block(tab, rk, win, x0 + 32 * jj);
          const uint4 vb = aes_ctr_run_block(tab, rk, win, x0 + 32 * jj + 32);
          noise_store(smem, o, base, b0 + 32 * jj, va);
          noise_store(smem, o, base, b0 + 32 * jj + 32, vb);
        }
      } else {
#pragma unroll 1
        for (uint32_t b = b0; b < nblk; b += 32)
          noise_store(smem, o, base, b, aes_ctr_run_block(tab, rk, win, x0 + (b - b0)));
      }
    }
  }
}

__global__ void __launch_bounds__(512, 1) k_noise(NoiseArgs a) {
  extern __shared__ uint32_t sT[];
  pdl_trigger();
  aes_fill_smem(sT, g_aes_img);
  if (a.tab_img) {
    // the context's prebuilt sampler table (k_noise_table's output)
    uint4 *d = reinterpret_cast<uint4 *>(sT + NOISE_TAB_OFF / 4);
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < 65536 / 16; i += blockDim.x) d[i] = a.tab_img[i];
  } else {
    noise_fill_table(sT + NOISE_TAB_OFF / 4, a);
  }
  __syncthreads();
  pdl_wait();
  const AesTab tab = aes_tab(sT);
  noise_runs(a, tab, reinterpret_cast<const char *>(sT),
             (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
             (uint64_t)gridDim.x * (blockDim.x >> 5));
}

LWE_BOUNDS_READER(lwe_bounds_read_kem)

// The sampler table exactly as k_noise builds and reads it, for all 65536
// words: out[w] = the sample of word w (a check of the table against the
// definition of the sampler; one CTA).
__global__ void __launch_bounds__(512, 1) k_noise_table(NoiseArgs a, int8_t *out) {
  extern __shared__ uint32_t sT[];
  noise_fill_table(sT + NOISE_TAB_OFF / 4, a);
  __syncthreads();
  const char *smem = reinterpret_cast<const char *>(sT);
  for (uint32_t w = threadIdx.x; w < 65536; w += blockDim.x) out[w] = (int8_t)tab_sample(smem, w);
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

// A S + E with A regenerated (KeyGen, Alg. 1, fused): persistent CTAs of
// 16 warps fill the AES tables once and walk the rows (warp per row, lane
// per 16-byte chunk = one AES block of A's counter layout).
__global__ void __launch_bounds__(512, 1) k_mul_as_fused(MulAsArgs a) {
  extern __shared__ uint32_t sT[];
  pdl_trigger();
  aes_fill_smem(sT, g_aes_img);
  __syncthreads();
  pdl_wait();
  const AesTab tab = aes_tab(sT);
  const uint32_t e = blockIdx.y;
  uint32_t key[4], rk[44];
  aes_load_key(a.seeds + (size_t)e * a.seed_stride, key);
  aes_key_expand(tab, key, rk);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = a.n;
  const uint32_t m = (1u << a.logq) - 1u, mm = m | (m << 16);
  const int8_t *St = a.St + (size_t)e * a.st_stride;
  const uint32_t rows = a.rows ? a.rows : n;
  for (uint32_t i = blockIdx.x * 16 + warp; i < rows; i += gridDim.x * 16) {
    int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // a lane's blocks step by 32 through the row: its 256-aligned counter
    // window (the first two AES rounds, aes_ctr_run) changes every 8 blocks
    AesCtrRun win;
    uint64_t wcur = ~0ull;
    for (uint32_t jc = lane; jc < n / 8; jc += 32) {
      const uint64_t b = (uint64_t)(a.row0 + i) * (n / 8) + jc;
      if ((b >> 8) != wcur) {
        wcur = b >> 8;
        win = aes_ctr_run(tab, rk, 0, b);
      }
      uint4 x = aes_ctr_run_block(tab, rk, win, (uint32_t)b & 255u);
      x.x &= mm;
      x.y &= mm;
      x.z &= mm;
      x.w &= mm;
      dot8_chunk(x, St, n, 8 * jc, acc);
    }
    warp_allreduce8(acc);
    if (lane == 0) {
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
}

// A S + E with stored A (KeyGen, Alg. 1).  A warp computes AS_ROWS rows of
// A together, so every 64-byte chunk of S^T it loads serves AS_ROWS rows,
// and keeps two 16-byte chunks of each row in flight per lane (A streams
// past L1; S^T stays there).  The 8 AS_ROWS partial sums of a lane are
// reduced across the warp by recursive halving, which leaves lane L with
// output L = (row L / 8, column L % 8) for one coalesced store.
#define AS_ROWS 4

LWE_DEV uint4 ld_stream_u4(const void *p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

LWE_DEV void dot8_rows(const uint4 *x, const int8_t *__restrict__ St, uint32_t n, uint32_t j,
                       int acc[AS_ROWS][8]) {
#pragma unroll
  for (int l = 0; l < 8; l++) {
    const uint2 s = ld_nc_u2(St + (size_t)l * n + j);
#pragma unroll
    for (int r = 0; r < AS_ROWS; r++) {
      acc[r][l] = __dp2a_lo((int)x[r].x, (int)s.x, acc[r][l]);
      acc[r][l] = __dp2a_hi((int)x[r].y, (int)s.x, acc[r][l]);
      acc[r][l] = __dp2a_lo((int)x[r].z, (int)s.y, acc[r][l]);
      acc[r][l] = __dp2a_hi((int)x[r].w, (int)s.y, acc[r][l]);
    }
  }
}

// Row groups (tasks) are dealt out task = CTA + grid * (warp + 8 k), so
// that with a grid of two CTAs per SM every SM streams the same share of A.
__global__ void __launch_bounds__(256) k_mul_as_rows(MulAsArgs a) {
  pdl_trigger();
  pdl_wait();
  const uint32_t e = blockIdx.y;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = a.n, nch = n / 8;
  const uint32_t tasks = (a.rows ? a.rows : n) / AS_ROWS;  // rows: a multiple of AS_ROWS
  const int8_t *St = a.St + (size_t)e * a.st_stride;
  for (uint32_t task = blockIdx.x + gridDim.x * warp; task < tasks; task += gridDim.x * 8) {
  const uint32_t i0 = task * AS_ROWS;
  if (!LWE_BOUNDS(i0 + AS_ROWS <= (a.rows ? a.rows : n), 109)) continue;
  const uint16_t *A0 = a.A + (size_t)e * a.a_stride + (size_t)i0 * n;
  int acc[AS_ROWS][8];
#pragma unroll
  for (int r = 0; r < AS_ROWS; r++)
#pragma unroll
    for (int l = 0; l < 8; l++) acc[r][l] = 0;
  for (uint32_t jc = lane; jc < nch; jc += 64) {
    const bool two = jc + 32 < nch;
    uint4 x0[AS_ROWS], x1[AS_ROWS];
#pragma unroll
    for (int r = 0; r < AS_ROWS; r++) x0[r] = ld_stream_u4(A0 + (size_t)r * n + 8 * (size_t)jc);
#pragma unroll
    for (int r = 0; r < AS_ROWS; r++)
      x1[r] = two ? ld_stream_u4(A0 + (size_t)r * n + 8 * (size_t)(jc + 32)) : make_uint4(0, 0, 0, 0);
    dot8_rows(x0, St, n, 8 * jc, acc);
    if (two) dot8_rows(x1, St, n, 8 * (jc + 32), acc);
  }
  // recursive halving: at offset o a lane keeps the half of its values
  // selected by lane bit o and adds the partner's copy of that half
  int v[32];
#pragma unroll
  for (int r = 0; r < AS_ROWS; r++)
#pragma unroll
    for (int l = 0; l < 8; l++) v[8 * r + l] = acc[r][l];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < o; j++) {
      const int send = up ? v[j] : v[j + o];
      const int keep = up ? v[j + o] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  const uint32_t r = lane >> 3, l = lane & 7, i = i0 + r;
  const uint32_t m = (1u << a.logq) - 1u;
  const int ev = a.E ? (int)a.E[(size_t)e * a.e_stride + (size_t)i * 8 + l] : 0;
  const uint16_t val = (uint16_t)((uint32_t)(v[0] + ev) & m);
  reinterpret_cast<uint16_t *>(a.out + (size_t)e * a.out_stride + 16 * (size_t)i)[l] = val;
  if (a.out2) reinterpret_cast<uint16_t *>(a.out2 + (size_t)e * a.out2_stride + 16 * (size_t)i)[l] = val;
  }
}

// The same for calls with few rows in all (one item, n up to a few
// thousand): the kernel above then has less than one row group per warp and
// each warp's chain of dependent loads sets the time.  Here a CTA takes one
// row group and its 8 warps split the columns, so 8 times as many warps keep
// loads in flight; their partial sums meet in shared memory.
__global__ void __launch_bounds__(256) k_mul_as_split(MulAsArgs a) {
  __shared__ int red[8][32];
  pdl_trigger();
  pdl_wait();
  const uint32_t e = blockIdx.y, i0 = blockIdx.x * AS_ROWS;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = a.n, nch = n / 8;
  const uint32_t c0 = warp * nch / 8, c1 = (warp + 1) * nch / 8;
  const int8_t *St = a.St + (size_t)e * a.st_stride;
  const uint16_t *A0 = a.A + (size_t)e * a.a_stride + (size_t)i0 * n;
  int acc[AS_ROWS][8];
#pragma unroll
  for (int r = 0; r < AS_ROWS; r++)
#pragma unroll
    for (int l = 0; l < 8; l++) acc[r][l] = 0;
  for (uint32_t jc = c0 + lane; jc < c1; jc += 64) {
    const bool two = jc + 32 < c1;
    uint4 x0[AS_ROWS], x1[AS_ROWS];
#pragma unroll
    for (int r = 0; r < AS_ROWS; r++) x0[r] = ld_stream_u4(A0 + (size_t)r * n + 8 * (size_t)jc);
#pragma unroll
    for (int r = 0; r < AS_ROWS; r++)
      x1[r] = two ? ld_stream_u4(A0 + (size_t)r * n + 8 * (size_t)(jc + 32)) : make_uint4(0, 0, 0, 0);
    dot8_rows(x0, St, n, 8 * jc, acc);
    if (two) dot8_rows(x1, St, n, 8 * (jc + 32), acc);
  }
  int v[32];
#pragma unroll
  for (int r = 0; r < AS_ROWS; r++)
#pragma unroll
    for (int l = 0; l < 8; l++) v[8 * r + l] = acc[r][l];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < o; j++) {
      const int send = up ? v[j] : v[j + o];
      const int keep = up ? v[j + o] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  red[warp][lane] = v[0];
  __syncthreads();
  if (warp != 0) return;
  int sum = 0;
#pragma unroll
  for (int w = 0; w < 8; w++) sum += red[w][lane];
  const uint32_t r = lane >> 3, l = lane & 7, i = i0 + r;
  const uint32_t m = (1u << a.logq) - 1u;
  const int ev = a.E ? (int)a.E[(size_t)e * a.e_stride + (size_t)i * 8 + l] : 0;
  const uint16_t val = (uint16_t)((uint32_t)(sum + ev) & m);
  reinterpret_cast<uint16_t *>(a.out + (size_t)e * a.out_stride + 16 * (size_t)i)[l] = val;
  if (a.out2) reinterpret_cast<uint16_t *>(a.out2 + (size_t)e * a.out2_stride + 16 * (size_t)i)[l] = val;
}

// Decrypt (Alg. 3): warp r of CTA e computes row r of M = C - B' S and the
// B message bits of its eight coefficients.
__global__ void __launch_bounds__(256) k_decrypt(DecryptArgs a) {
  pdl_trigger();
  pdl_wait();
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

// S' A (+ E') for one or more items on the CUDA cores (Alg. 2), A stored
// (LDG.128 of 8 columns per row) or regenerated (one AES block per row and
// 8 columns, the counter layout of A).  CTA = (256-column block, row
// split, item): lane l owns columns 8 l .. 8 l + 7 of the block, warp w the
// row pairs (2p, 2p + 1) with p = w (mod 8); the pair's S' bytes are staged
// in shared memory so that one dp2a multiplies two rows.  The warps' sums
// meet in shared memory; when a call has few items the rows are split over
// a cluster of R CTAs whose partial sums are added through distributed
// shared memory, so no global workspace is needed.  Then E' is added and
// the row stored, or (CMP) compared with the received ciphertext.
#define SA_PAIRS 512  // row pairs of S' staged at a time (8 KB)

LWE_DEV uint32_t cluster_map(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
LWE_DEV int ld_cluster_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
LWE_DEV void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// word q of pair p: S'[2q][2p], S'[2q][2p+1], S'[2q+1][2p], S'[2q+1][2p+1]
LWE_DEV void sa_stage(const int8_t *S, uint32_t n, uint32_t c0, uint32_t cn, uint4 *sP,
                      uint32_t tid, uint32_t nt) {
  for (uint32_t q = tid; q < cn; q += nt) {
    const uint32_t i = 2 * (c0 + q);
    uint32_t w[4];
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
      const uint32_t lo = *reinterpret_cast<const uint16_t *>(S + (size_t)(2 * kk) * n + i);
      const uint32_t hi = *reinterpret_cast<const uint16_t *>(S + (size_t)(2 * kk + 1) * n + i);
      w[kk] = lo | (hi << 16);
    }
    sP[q] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// One column c of both rows of a pair as two 16-bit halves, times the pair's
// S' bytes for all 8 rows k: acc[k] += S'[k][2p] A[2p][c] + S'[k][2p+1] A[2p+1][c]
LWE_DEV void sa_mac_col(int pk, const uint4 sp, int *acc_c /* [8] stride */, int stride) {
  const uint32_t sw[4] = {sp.x, sp.y, sp.z, sp.w};
#pragma unroll
  for (int q = 0; q < 4; q++) {
    acc_c[(2 * q) * stride] = __dp2a_lo(pk, (int)sw[q], acc_c[(2 * q) * stride]);
    acc_c[(2 * q + 1) * stride] = __dp2a_hi(pk, (int)sw[q], acc_c[(2 * q + 1) * stride]);
  }
}

// The CTA's (and with R > 1 the cluster's) sums red[k][c][32] (column
// 8 lane + c of the block) are finished: + E', mod q, store or compare.
template <bool CMP>
LWE_DEV void sa_epilogue(const MulSaArgs &a, int *red, uint32_t cb, uint32_t rsplit, uint32_t R,
                         uint32_t e, uint32_t tid, uint32_t nt) {
  const uint32_t n = a.n, mq = (1u << a.logq) - 1u;
  const uint32_t share = 2048 / R;
  uint32_t diff = 0;
  for (uint32_t v = rsplit * share + tid; v < (rsplit + 1) * share; v += nt) {
    const uint32_t k = v >> 8, col = v & 255;
    const uint32_t idx = k * 256 + (col & 7) * 32 + (col >> 3);
    int sum = 0;
    if (R > 1) {
      for (uint32_t r = 0; r < R; r++) sum += ld_cluster_s32(cluster_map(red + idx, r));
    } else {
      sum = red[idx];
    }
    const uint32_t j = cb * 256 + col;
    if (j < n) {
      if (a.E) sum += a.E[(size_t)e * a.e_stride + (size_t)k * n + j];
      const uint32_t val = (uint32_t)sum & mq;
      uint16_t *o = reinterpret_cast<uint16_t *>(a.out + (size_t)e * a.out_stride) + (size_t)k * n + j;
      if (CMP)
        diff |= val ^ (uint32_t)*o;
      else
        *o = (uint16_t)val;
    }
  }
  if (CMP) {
    diff = __reduce_or_sync(0xffffffffu, diff);
    if ((tid & 31) == 0 && diff) atomicOr(a.flags + e, 1u);
  }
}

template <bool CMP>
__global__ void __launch_bounds__(256) k_sa(MulSaArgs a) {
  extern __shared__ uint4 sm4[];
  pdl_trigger();
  pdl_wait();
  uint4 *sP = sm4;
  int *red = reinterpret_cast<int *>(sm4 + SA_PAIRS);
  const uint32_t cb = blockIdx.x, rsplit = blockIdx.y, R = gridDim.y, e = blockIdx.z;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t n = a.n;
  const uint32_t j0 = cb * 256 + 8 * lane;
  const bool jv = j0 < n;  // n and j0 are multiples of 8: a chunk is all in or all out
  for (uint32_t i = tid; i < 2048; i += 256) red[i] = 0;
  const int8_t *S = a.S + (size_t)e * a.s_stride;
  const uint32_t p0 = a.row0 / 2, p1 = (a.row1 ? a.row1 : n) / 2;
  // a stored row block starts at row row0
  const uint16_t *Aitem = a.A_ptrs ? a.A_ptrs[e] : a.A;
  const uint32_t r0 = a.row0;
  const uint32_t per = (p1 - p0 + R - 1) / R;
  const uint32_t pb = min(p1, p0 + rsplit * per), pe = min(p1, pb + per);
  int acc[8][8];
#pragma unroll
  for (int k = 0; k < 8; k++)
#pragma unroll
    for (int c = 0; c < 8; c++) acc[k][c] = 0;
  auto row_chunk = [&](uint32_t i) -> uint4 {
    return jv && LWE_BOUNDS(i >= r0 && i < (a.row1 ? a.row1 : n), 110)
               ? ld_nc_u4(Aitem + (size_t)(i - r0) * n + j0)
               : make_uint4(0, 0, 0, 0);
  };
  auto mac_pair = [&](const uint4 x0, const uint4 x1, const uint4 sp) {
    const uint32_t w0[4] = {x0.x, x0.y, x0.z, x0.w}, w1[4] = {x1.x, x1.y, x1.z, x1.w};
#pragma unroll
    for (int c = 0; c < 8; c++) {
      // column c of both rows as two 16-bit halves (signed: same residues)
      const int pk = (int)__byte_perm(w0[c >> 1], w1[c >> 1], (c & 1) ? 0x7632 : 0x5410);
      sa_mac_col(pk, sp, &acc[0][c], 8);
    }
  };
  for (uint32_t c0 = pb; c0 < pe; c0 += SA_PAIRS) {
    const uint32_t cn = min((uint32_t)SA_PAIRS, pe - c0);
    __syncthreads();
    sa_stage(S, n, c0, cn, sP, tid, 256);
    __syncthreads();
    uint32_t q = warp;
    for (; q + 24 < cn; q += 32) {  // four pairs (eight rows) in flight
      const uint32_t i = 2 * (c0 + q);
      uint4 x[8];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        x[2 * u] = row_chunk(i + 16 * u);
        x[2 * u + 1] = row_chunk(i + 16 * u + 1);
      }
#pragma unroll
      for (int u = 0; u < 4; u++) mac_pair(x[2 * u], x[2 * u + 1], sP[q + 8 * u]);
    }
    for (; q + 8 < cn; q += 16) {  // two pairs in flight
      const uint32_t i = 2 * (c0 + q), i2 = i + 16;
      const uint4 x0 = row_chunk(i), x1 = row_chunk(i + 1);
      const uint4 y0 = row_chunk(i2), y1 = row_chunk(i2 + 1);
      mac_pair(x0, x1, sP[q]);
      mac_pair(y0, y1, sP[q + 8]);
    }
    if (q < cn) {
      const uint32_t i = 2 * (c0 + q);
      mac_pair(row_chunk(i), row_chunk(i + 1), sP[q]);
    }
  }
  // the CTA's sum: red[k][c][lane] (column 8 lane + c)
#pragma unroll
  for (int k = 0; k < 8; k++)
#pragma unroll
    for (int c = 0; c < 8; c++) atomicAdd(&red[k * 256 + c * 32 + lane], acc[k][c]);
  __syncthreads();
  if (R > 1) cluster_barrier();  // every CTA of the cluster has its partial sum
  sa_epilogue<CMP>(a, red, cb, rsplit, R, e, tid, 256);
  if (R > 1) cluster_barrier();  // no CTA leaves while others read its shared memory
}

// The same product with A regenerated (the AES tables in shared memory): 16
// warps; a lane pair shares one 8-column chunk, lane s of the pair
// encrypting row 2p + s of each row pair and the two swapping half blocks,
// so each lane holds 4 columns of both rows (32 sums, room for 16 warps).
// Warps 0-7 take columns 0-127 of the CTA's block, warps 8-15 columns
// 128-255.
template <bool CMP>
__global__ void __launch_bounds__(512, 1) k_sa_fused(MulSaArgs a) {
  extern __shared__ uint4 sm4[];
  uint8_t *base = reinterpret_cast<uint8_t *>(sm4);
  uint4 *sP = reinterpret_cast<uint4 *>(base + AES_SMEM_BYTES);
  int *red = reinterpret_cast<int *>(base + AES_SMEM_BYTES + SA_PAIRS * 16);
  const uint32_t cb = blockIdx.x, rsplit = blockIdx.y, R = gridDim.y, e = blockIdx.z;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rw = warp & 7, half = warp >> 3, s = lane & 1;
  const uint32_t n = a.n;
  const uint32_t chunk = cb * 32 + half * 16 + (lane >> 1);  // 8-column chunk index
  const uint32_t j0 = 8 * chunk;
  const bool jv = j0 < n;
  pdl_trigger();
  for (uint32_t i = tid; i < 2048; i += 512) red[i] = 0;
  uint32_t *sT = reinterpret_cast<uint32_t *>(base);
  aes_fill_smem(sT, g_aes_img);
  __syncthreads();
  pdl_wait();
  const AesTab tab = aes_tab(sT);
  uint32_t key[4], rk[44];
  aes_load_key(a.seed_ptrs ? a.seed_ptrs[e] + a.seed_off : a.seedA, key);
  aes_key_expand(tab, key, rk);
  const uint32_t mq = (1u << a.logq) - 1u, mm = mq | (mq << 16);
  const int8_t *S = a.S + (size_t)e * a.s_stride;
  const uint32_t p0 = a.row0 / 2, p1 = (a.row1 ? a.row1 : n) / 2;
  const uint32_t per = (p1 - p0 + R - 1) / R;
  const uint32_t pb = min(p1, p0 + rsplit * per), pe = min(p1, pb + per);
  int acc[8][4];
#pragma unroll
  for (int k = 0; k < 8; k++)
#pragma unroll
    for (int c = 0; c < 4; c++) acc[k][c] = 0;
  for (uint32_t c0 = pb; c0 < pe; c0 += SA_PAIRS) {
    const uint32_t cn = min((uint32_t)SA_PAIRS, pe - c0);
    __syncthreads();
    sa_stage(S, n, c0, cn, sP, tid, 512);
    __syncthreads();
    for (uint32_t q = rw; q < cn; q += 8) {
      const uint32_t i = 2 * (c0 + q) + s;  // this lane's row of the pair
      uint4 x = make_uint4(0, 0, 0, 0);
      if (jv) {
        x = aes_ctr_block(tab, rk, 0, (uint64_t)i * (n / 8) + chunk);
        x.x &= mm;
        x.y &= mm;
        x.z &= mm;
        x.w &= mm;
      }
      // lane 0 of the pair keeps columns 0-3 of its row and takes columns
      // 0-3 of row 2p+1; lane 1 keeps columns 4-7 of row 2p+1 and takes 4-7
      // of row 2p
      const uint32_t g0 = s ? x.x : x.z, g1 = s ? x.y : x.w;
      const uint32_t r0 = __shfl_xor_sync(0xffffffffu, g0, 1);
      const uint32_t r1 = __shfl_xor_sync(0xffffffffu, g1, 1);
      const uint32_t a0 = s ? r0 : x.x, a1 = s ? r1 : x.y;  // row 2p, my 4 columns
      const uint32_t b0 = s ? x.z : r0, b1 = s ? x.w : r1;  // row 2p+1
      const uint4 sp = sP[q];
      sa_mac_col((int)__byte_perm(a0, b0, 0x5410), sp, &acc[0][0], 4);
      sa_mac_col((int)__byte_perm(a0, b0, 0x7632), sp, &acc[0][1], 4);
      sa_mac_col((int)__byte_perm(a1, b1, 0x5410), sp, &acc[0][2], 4);
      sa_mac_col((int)__byte_perm(a1, b1, 0x7632), sp, &acc[0][3], 4);
    }
  }
  // column of the block owned by (half, lane): 128 half + 8 (lane / 2) + 4 s + c
  const uint32_t cl = half * 16 + (lane >> 1);  // chunk within the block (0..31)
#pragma unroll
  for (int k = 0; k < 8; k++)
#pragma unroll
    for (int c = 0; c < 4; c++) atomicAdd(&red[k * 256 + (4 * s + c) * 32 + cl], acc[k][c]);
  __syncthreads();
  if (R > 1) cluster_barrier();
  sa_epilogue<CMP>(a, red, cb, rsplit, R, e, tid, 512);
  if (R > 1) cluster_barrier();
}

// ---------------------------------------------------------------------------
// V = S' B + E'' and C = V + Enc(mu) (Alg. 2); CTA per item, warp per row k.
// ---------------------------------------------------------------------------
template <bool CMP>
__global__ void __launch_bounds__(256) k_v_encode(VEncArgs a) {
  pdl_trigger();
  pdl_wait();
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
  pdl_trigger();
  pdl_wait();
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
// K' and seedSE' do not depend on each other: a CTA of two warps takes 32
// items, warp 0 computing K' and warp 1 seedSE' and its key schedule (both
// warps hash mu themselves), so each item waits for two permutations in
// Encaps and one in Decaps instead of three and two.
__global__ void __launch_bounds__(64) k_derive(DeriveArgs a) {
  __shared__ uint32_t sT0[256];  // the key expansion's S-box lookups stay on chip
  pdl_trigger();
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) sT0[i] = g_aes_T0[i];
  __syncthreads();
  pdl_wait();
  const uint32_t w = threadIdx.x >> 5;
  const uint32_t e = blockIdx.x * 32 + (threadIdx.x & 31);
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
      if (w == 0) mu64[i] = x[4 + i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; i++) x[4 + i] = (uint32_t)i < nb ? mu64[i] : 0;
  }
  const uint8_t *pkh = a.pkh_ptrs ? a.pkh_ptrs[e] + a.pkh_off : a.pkh + (size_t)e * a.pkh_stride;
  load32_le(pkh, x);
  // (every lane is written unconditionally with a selected value: a
  // conditional store to lane 4 + nb would become a dynamically indexed
  // state, i.e. local memory)
  if (w == 0) {
    // K' = H(pkh || mu): 32 + 8 nb bytes, padding opens lane 4 + nb
#pragma unroll
    for (int i = 0; i < 25; i++) s[i] = i < 8 ? x[i] : 0;
#pragma unroll
    for (int i = 5; i < 9; i++) s[i] ^= (uint32_t)i == 4 + nb ? 0x06ull : 0ull;
    s[SHA3_RATE / 8 - 1] ^= 0x8000000000000000ull;
    keccak_f1600(s);
    sha3_digest(s, a.kprime + 32 * (size_t)e);
    return;
  }
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

// ---------------------------------------------------------------------------
// The same hashes with one Keccak state per warp (keccak_warp.cuh), for
// launches of few items: one permutation then takes one warp ~1.5-2.7 us
// instead of one thread ~5.6 us, and independent hashes of an item run in
// different warps.  Thread t builds lane t of the padded single-block
// message; lanes 0..3 of the result are the digest.
// ---------------------------------------------------------------------------
LWE_DEV uint64_t ld_le64(const uint8_t *p) {
  if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) return *reinterpret_cast<const uint64_t *>(p);
  uint64_t v = 0;
#pragma unroll
  for (int b = 0; b < 8; b++) v |= (uint64_t)p[b] << (8 * b);
  return v;
}

LWE_DEV void st_le64(uint8_t *p, uint64_t v) {
#pragma unroll
  for (int b = 0; b < 8; b++) p[b] = (uint8_t)(v >> (8 * b));
}

// lane t of prefix || 32 bytes, padded: the 32 bytes shifted up one byte,
// the padding opening byte 1 of lane 4
LWE_DEV uint64_t prefixed32_lane(uint8_t prefix, const uint8_t *msg32, uint32_t t) {
  uint64_t v = 0;
  if (t < 4) v = ld_le64(msg32 + 8 * t) << 8;
  if (t >= 1 && t <= 4) v |= ld_le64(msg32 + 8 * (t - 1)) >> 56;
  if (t == 0) v |= prefix;
  if (t == 4) v |= 0x0600ull;
  if (t == SHA3_RATE / 8 - 1) v ^= 0x8000000000000000ull;
  return v;
}

// KeyGen seeds (Alg. 1): warp j of the item's CTA hashes prefix j || ms
__global__ void __launch_bounds__(96) k_keygen_seeds_warp(KeygenSeedArgs a) {
  __shared__ uint32_t sT0[256];
  pdl_trigger();
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) sT0[i] = g_aes_T0[i];
  __syncthreads();
  pdl_wait();
  const uint32_t e = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31, t = lane % 25;
  const KeccakWarpMap km = keccak_warp_map(lane);
  const uint8_t prefix = w == 0 ? 0x41 : (w == 1 ? 0x53 : 0x5A);
  const uint64_t v = keccak_f1600_warp(km, prefixed32_lane(prefix, a.ms + 32 * (size_t)e, t));
  uint8_t *pk = a.pk + (size_t)e * a.pk_bytes;
  uint8_t *sk = a.sk + (size_t)e * a.sk_bytes;
  uint8_t *ws = a.ws_seeds + 32 * (size_t)e;
  if (w == 0) {  // seedA
    if (lane < 2) {
      st_le64(pk + 8 * lane, v);
      st_le64(sk + a.sk_pk_off + 8 * lane, v);
      st_le64(ws + 8 * lane, v);
    }
  } else if (w == 1) {  // seedSE and its key schedule
    if (lane < 2) st_le64(ws + 16 + 8 * lane, v);
    const uint64_t v1 = shfl64(v, 1);
    if (lane == 0) {
      const uint32_t key[4] = {(uint32_t)v, (uint32_t)(v >> 32), (uint32_t)v1, (uint32_t)(v1 >> 32)};
      uint32_t rk[44];
      aes_key_expand_global(sT0, key, rk);
      uint4 *dst = reinterpret_cast<uint4 *>(a.ws_rk + 44 * (size_t)e);
#pragma unroll
      for (int i = 0; i < 11; i++)
        dst[i] = make_uint4(rk[4 * i], rk[4 * i + 1], rk[4 * i + 2], rk[4 * i + 3]);
    }
  } else if (lane < 4) {  // z
    st_le64(sk + a.sk_z_off + 8 * lane, v);
  }
}

// Encaps / Decaps derivation (Alg. 4, 5): both warps of the item's CTA
// hash mu (Encaps), then warp 0 K' = H(pkh || mu) and warp 1
// seedSE' = H(0x01 || pkh || mu) with its key schedule
__global__ void __launch_bounds__(64, 1) k_derive_warp(DeriveArgs a) {
  __shared__ uint32_t sT0[256];
  pdl_trigger();
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) sT0[i] = g_aes_T0[i];
  __syncthreads();
  pdl_wait();
  const uint32_t e = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31, t = lane % 25;
  const KeccakWarpMap km = keccak_warp_map(lane);
  const uint32_t nb = a.mu_bytes / 8;  // lanes of mu, 1..4
  uint64_t *mu64 = reinterpret_cast<uint64_t *>(a.mu + 32 * (size_t)e);
  uint64_t mu_l = 0;  // lane t < 4: lane t of mu (zero beyond nb)
  if (a.coins) {
    const uint64_t v = keccak_f1600_warp(km, prefixed32_lane(0x4D, a.coins + 32 * (size_t)e, t));
    mu_l = t < nb ? v : 0;
    if (w == 0 && lane < 4) mu64[lane] = mu_l;
  } else if (t < nb) {
    mu_l = mu64[t];
  }
  // x = pkh (4 lanes) || mu (4 lanes) || zeros; thread t holds x[t]
  const uint8_t *pkh = a.pkh_ptrs ? a.pkh_ptrs[e] + a.pkh_off : a.pkh + (size_t)e * a.pkh_stride;
  const uint64_t mu_at = shfl64(mu_l, (lane - 4) & 31);
  const uint64_t x = t < 4 ? ld_le64(pkh + 8 * t) : (t < 8 ? mu_at : 0);
  if (w == 0) {
    uint64_t m = x;
    if (t == 4 + nb) m ^= 0x06ull;
    if (t == SHA3_RATE / 8 - 1) m ^= 0x8000000000000000ull;
    const uint64_t v = keccak_f1600_warp(km, m);
    if (lane < 4) st_le64(a.kprime + 32 * (size_t)e + 8 * lane, v);
    return;
  }
  const uint64_t xp = shfl64(x, (lane + 31) & 31);  // x[t - 1]
  uint64_t m = t == 0 ? (0x01ull | (x << 8)) : ((xp >> 56) | (x << 8));
  if (t == 4 + nb) m ^= 0x0600ull;
  if (t == SHA3_RATE / 8 - 1) m ^= 0x8000000000000000ull;
  const uint64_t v = keccak_f1600_warp(km, m);
  if (lane < 2) st_le64(a.seeds + 32 * (size_t)e + 8 * lane, v);
  const uint64_t v1 = shfl64(v, 1);
  if (lane == 0) {
    const uint32_t key[4] = {(uint32_t)v, (uint32_t)(v >> 32), (uint32_t)v1, (uint32_t)(v1 >> 32)};
    uint32_t rk[44];
    aes_key_expand_global(sT0, key, rk);
    uint4 *dst = reinterpret_cast<uint4 *>(a.rk + 44 * (size_t)e);
#pragma unroll
    for (int i = 0; i < 11; i++)
      dst[i] = make_uint4(rk[4 * i], rk[4 * i + 1], rk[4 * i + 2], rk[4 * i + 3]);
  }
}

// Decaps key (Alg. 5): K = H(K' || H(c)) when the re-encryption matched,
// else H(z || H(c)); one warp per item
__global__ void __launch_bounds__(32) k_final_key_warp(FinalKeyArgs a) {
  pdl_trigger();
  pdl_wait();
  const uint32_t e = blockIdx.x, lane = threadIdx.x, t = lane % 25;
  const KeccakWarpMap km = keccak_warp_map(lane);
  const uint32_t f = a.flags[e];
  const uint64_t keep = (uint64_t)0 - (uint64_t)(((f | (0u - f)) >> 31) ^ 1u);
  uint64_t m = 0;
  if (t < 4) {
    const uint64_t *kp = reinterpret_cast<const uint64_t *>(a.kprime + 32 * (size_t)e);
    const uint64_t *z =
        reinterpret_cast<const uint64_t *>(a.z_ptrs ? a.z_ptrs[e] + a.z_off : a.z);
    m = (kp[t] & keep) | (z[t] & ~keep);
  } else if (t < 8) {
    m = reinterpret_cast<const uint64_t *>(a.hc + 32 * (size_t)e)[t - 4];
  }
  if (t == 8) m ^= 0x06ull;
  if (t == SHA3_RATE / 8 - 1) m ^= 0x8000000000000000ull;
  const uint64_t v = keccak_f1600_warp(km, m);
  if (lane < 4) st_le64(a.K + 32 * (size_t)e + 8 * lane, v);
}

// Tree hash: tpi threads per message compute its 1024-byte-chunk digests
// into shared memory; threads 0..ipc-1 (one per message, so the root phase
// fills whole warps) then hash the digests -- the root -- and, for Encaps,
// derive the key.  A message's digests sit at a stride of 4 m + 1 words so
// the root threads' 64-bit reads fall in different banks.
__global__ void __launch_bounds__(TREE_MAX_THREADS) k_tree(TreeArgs a) {
  extern __shared__ uint64_t sleaf[];  // [ipc][4 m + 1]
  pdl_trigger();
  pdl_wait();
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
        if (!LWE_BOUNDS(off < a.len, 106)) continue;
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

// Tree hash of batches whose full-length leaves need 13 warps per CTA (one
// CTA per SM; e.g. 4096 ciphertexts of n = 976: 27 per CTA, 405 leaves of
// 8 permutations).  With one leaf per thread, 13 leaf warps put 4 warps on
// one SM sub-partition (SMSP) and 3 on the others: the loaded one needs 32
// warp-permutations where the others need 24, and the roots then run alone.
// Here, 16 warps with fixed roles:
//   - warps 0, 4, 8, 12 (SMSP 0) take the 128 leaves with the highest chunk
//     indices and run only TB_SPLIT of their 8 permutations; their sponge
//     states go to shared memory ([25][128] words);
//   - the nine other leaf warps (3 per SMSP 1-3) take the remaining leaves
//     whole;
//   - helper warps 14 and 15 (SMSPs 2, 3) finish the leaves of SMSP 0, two
//     warps' worth each, once those have stopped;
//   - warp 13 (SMSP 1) hashes the short last chunk of every message, then
//     the root: the root's first blocks absorb digests of low chunk indices,
//     which all come from SMSPs 1-3, so they run while the helpers work;
//     the rest of the root (and the Encaps key) follows the helpers.
// Named barriers (fixed thread counts, every warp meets each of its
// barriers exactly once): 1 leaf warps of SMSPs 1-3 -> warp 13 (320);
// 2 warps 0, 4 -> helper 14 (96); 4 warps 8, 12 -> helper 15 (96);
// 3 helpers -> warp 13 (96).  At most 96 registers per thread (no spills):
// a CTA then leaves room in the SM's register file for the CTAs of Decaps'
// small kernels, which run beside its H(c) on the other stream.
#define TB_SPLIT 6
#define TB_SLOTS 128

LWE_DEV void bar_arrive(uint32_t id, uint32_t n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
LWE_DEV void bar_sync(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__global__ void __maxnreg__(96) k_tree_bal(TreeArgs a) {
  extern __shared__ uint64_t sm[];
  pdl_trigger();
  pdl_wait();
  const uint32_t words = 4 * a.m + 1;
  uint64_t *sdig = sm;                              // [ipc][4 m + 1]
  uint64_t *shand = sm + (size_t)a.ipc * words;     // [25][TB_SLOTS]
  const uint32_t e0 = blockIdx.x * a.ipc;
  const uint32_t nmsg = min(a.ipc, a.count - e0);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ML = a.ml;                         // full-length chunks per message
  const uint32_t NL = nmsg * ML;
  const uint32_t fullp = LWE_TREE_CHUNK / SHA3_RATE + 1;  // permutations per full chunk
  uint64_t s[25];
  auto msg_of = [&](uint32_t li) -> const uint8_t * {
    const uint32_t e = e0 + li;
    return a.msg_ptrs ? a.msg_ptrs[e] : a.msgs + (size_t)e * a.stride;
  };
  // leaf k (k < NL): chunk ML - 1 - k / nmsg of message k % nmsg, so the
  // first TB_SLOTS leaves are the highest chunk indices
  auto put_digest = [&](uint32_t li, uint32_t c, const uint64_t *st) {
    if (!LWE_BOUNDS(li < nmsg && c < a.m, 102)) return;
    uint64_t *d = sdig + (size_t)li * words + 4 * c;
    d[0] = st[0];
    d[1] = st[1];
    d[2] = st[2];
    d[3] = st[3];
  };
  if (warp < 13 && (warp & 3) == 0) {
    // SMSP 0: the first TB_SPLIT permutations of leaves 0 .. TB_SLOTS-1
    const uint32_t k = 32 * (warp >> 2) + lane;
    if (k < NL && LWE_BOUNDS(k < TB_SLOTS, 101)) {
      const uint32_t li = k % nmsg, c = ML - 1 - k / nmsg;
      sha3_init(s);
      if (LWE_BOUNDS((c + 1) * LWE_TREE_CHUNK <= a.len, 103))
        sha3_absorb_global(msg_of(li) + (size_t)c * LWE_TREE_CHUNK, LWE_TREE_CHUNK, 0, TB_SPLIT, s);
#pragma unroll
      for (int i = 0; i < 25; i++) shand[i * TB_SLOTS + k] = s[i];
    }
    __syncwarp();
    bar_arrive(warp < 8 ? 2 : 4, 96);
  } else if (warp < 13) {
    // SMSPs 1-3: whole leaves TB_SLOTS ..
    const uint32_t idx = warp - 1 - (warp >> 2);  // 0 .. 8
    const uint32_t k = TB_SLOTS + 32 * idx + lane;
    if (k < NL) {
      const uint32_t li = k % nmsg, c = ML - 1 - k / nmsg;
      sha3_init(s);
      if (LWE_BOUNDS((c + 1) * LWE_TREE_CHUNK <= a.len, 103))
        sha3_absorb_global(msg_of(li) + (size_t)c * LWE_TREE_CHUNK, LWE_TREE_CHUNK, 0, fullp, s);
      put_digest(li, c, s);
    }
    __syncwarp();
    bar_arrive(1, 320);
  } else if (warp >= 14) {
    // helpers: the last permutations of two SMSP-0 warps' leaves each
    bar_sync(warp == 14 ? 2 : 4, 96);
    for (uint32_t g = 0; g < 2; g++) {
      const uint32_t k = 32 * (2 * (warp - 14) + g) + lane;
      if (k < NL && LWE_BOUNDS(k < TB_SLOTS, 104)) {
        const uint32_t li = k % nmsg, c = ML - 1 - k / nmsg;
#pragma unroll
        for (int i = 0; i < 25; i++) s[i] = shand[i * TB_SLOTS + k];
        sha3_absorb_global(msg_of(li) + (size_t)c * LWE_TREE_CHUNK, LWE_TREE_CHUNK, TB_SPLIT,
                           fullp, s);
        put_digest(li, c, s);
      }
    }
    __syncwarp();
    bar_arrive(3, 96);
  } else {
    // warp 13: the short last chunks, then the roots (and Encaps' key)
    const uint32_t li = lane;
    const bool mine = li < nmsg;
    if (mine && ML < a.m) {
      const uint32_t c = a.m - 1, off = c * LWE_TREE_CHUNK, len = a.len - off;
      sha3_init(s);
      if (LWE_BOUNDS(off < a.len && len <= LWE_TREE_CHUNK, 105))
        sha3_absorb_global(msg_of(li) + off, len, 0, len / SHA3_RATE + 1, s);
      put_digest(li, c, s);
    }
    // root blocks whose digests all come from chunks below the lowest
    // chunk index held by SMSP 0 are absorbed before the helpers finish
    const uint32_t held = min((uint32_t)TB_SLOTS, NL);
    const uint32_t cmin = held ? ML - 1 - (held - 1) / nmsg : a.m;
    const uint32_t rlen = 32 * a.m, nb = rlen / SHA3_RATE + 1;
    uint32_t early = 0;
    while (early < nb && min(rlen - 1, SHA3_RATE * early + SHA3_RATE - 1) / 32 < cmin) early++;
    __syncwarp();
    bar_sync(1, 320);
    const uint8_t *root = reinterpret_cast<const uint8_t *>(sdig + (size_t)li * words);
    sha3_init(s);
    if (mine) sha3_absorb_mem(root, rlen, 0, early, s);
    __syncwarp();
    bar_sync(3, 96);
    if (mine) {
      sha3_absorb_mem(root, rlen, early, nb, s);
      const uint32_t e = e0 + li;
      if (a.mode == TREE_DIGEST) {
        sha3_digest(s, a.out + (size_t)e * a.out_stride);
        if (a.out2) sha3_digest(s, a.out2 + (size_t)e * a.out2_stride);
      } else {
        // Encaps (Alg. 4): K = H(K' || H(c))
        uint64_t lanes[SHA3_RATE / 8];
        lanes_zero(lanes);
        const uint64_t *kp = reinterpret_cast<const uint64_t *>(a.kprime + 32 * (size_t)e);
        for (int i = 0; i < 4; i++) lanes[i] = kp[i];
        for (int i = 0; i < 4; i++) lanes[4 + i] = s[i];
        sha3_256_lanes(lanes, 64, s);
        sha3_digest(s, a.out + 32 * (size_t)e);
      }
    }
  }
}

// Tree hash of batches whose full-length leaves fill at most 12 warps per
// CTA (e.g. 4096 ciphertexts of n = 640: 27 per SM, 270 leaves): the leaves
// are packed densely, leaf k on warp k / 32 of warps 0-11, so consecutive
// warps fall on consecutive SM sub-partitions and every SMSP holds
// floor or ceil of WL / 4 leaf warps (k_tree instead gives each message a
// power-of-two group of threads, which leaves lanes idle).  The short last
// chunks and then the roots (and Encaps' key) run on one warp of the SMSP
// with the fewest leaf warps, `rw`.  One named barrier: the twelve leaf
// warps (whether or not they hold leaves) -> the root warp (416 threads).
__global__ void __maxnreg__(96) k_tree_dense(TreeArgs a) {
  extern __shared__ uint64_t sm[];
  pdl_trigger();
  pdl_wait();
  const uint32_t words = 4 * a.m + 1;
  uint64_t *sdig = sm;  // [ipc][4 m + 1]
  const uint32_t e0 = blockIdx.x * a.ipc;
  const uint32_t nmsg = min(a.ipc, a.count - e0);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ML = a.ml, NL = nmsg * ML;
  const uint32_t fullp = LWE_TREE_CHUNK / SHA3_RATE + 1;
  uint64_t s[25];
  auto msg_of = [&](uint32_t li) -> const uint8_t * {
    const uint32_t e = e0 + li;
    return a.msg_ptrs ? a.msg_ptrs[e] : a.msgs + (size_t)e * a.stride;
  };
  auto put_digest = [&](uint32_t li, uint32_t c, const uint64_t *st) {
    if (!LWE_BOUNDS(li < nmsg && c < a.m, 111)) return;
    uint64_t *d = sdig + (size_t)li * words + 4 * c;
    d[0] = st[0];
    d[1] = st[1];
    d[2] = st[2];
    d[3] = st[3];
  };
  if (warp < 12) {
    const uint32_t k = 32 * warp + lane;  // leaf k: chunk k % ML of message k / ML
    if (k < NL) {
      const uint32_t li = k / ML, c = k % ML;
      sha3_init(s);
      if (LWE_BOUNDS((c + 1) * LWE_TREE_CHUNK <= a.len, 112))
        sha3_absorb_global(msg_of(li) + (size_t)c * LWE_TREE_CHUNK, LWE_TREE_CHUNK, 0, fullp, s);
      put_digest(li, c, s);
    }
    __syncwarp();
    bar_arrive(1, 416);
    return;
  }
  if (warp != a.rw) return;
  const uint32_t li = lane;
  const bool mine = li < nmsg;
  if (mine && ML < a.m) {
    const uint32_t c = a.m - 1, off = c * LWE_TREE_CHUNK, len = a.len - off;
    sha3_init(s);
    if (LWE_BOUNDS(off < a.len && len <= LWE_TREE_CHUNK, 113))
      sha3_absorb_global(msg_of(li) + off, len, 0, len / SHA3_RATE + 1, s);
    put_digest(li, c, s);
  }
  __syncwarp();
  bar_sync(1, 416);
  if (!mine) return;
  const uint32_t rlen = 32 * a.m;
  sha3_init(s);
  sha3_absorb_mem(reinterpret_cast<const uint8_t *>(sdig + (size_t)li * words), rlen, 0,
                  rlen / SHA3_RATE + 1, s);
  const uint32_t e = e0 + li;
  if (a.mode == TREE_DIGEST) {
    sha3_digest(s, a.out + (size_t)e * a.out_stride);
    if (a.out2) sha3_digest(s, a.out2 + (size_t)e * a.out2_stride);
  } else {
    // Encaps (Alg. 4): K = H(K' || H(c))
    uint64_t lanes[SHA3_RATE / 8];
    lanes_zero(lanes);
    const uint64_t *kp = reinterpret_cast<const uint64_t *>(a.kprime + 32 * (size_t)e);
    for (int i = 0; i < 4; i++) lanes[i] = kp[i];
    for (int i = 0; i < 4; i++) lanes[4 + i] = s[i];
    sha3_256_lanes(lanes, 64, s);
    sha3_digest(s, a.out + 32 * (size_t)e);
  }
}

// Tree hash with one Keccak state per warp (keccak_warp.cuh), for launches
// of few messages, where one state per thread would leave the GPU idle
// behind a chain of sequential permutations.  A thread-block cluster of Q
// CTAs (W warps each, on Q SMs, so that few warps share an SM's shuffle
// unit) takes one message: warp w of CTA q hashes chunks qW + w, qW + w +
// QW, ... and stores each digest in the shared memory of the cluster's
// first CTA, whose warp 0 then hashes the digests (the root) and, for
// Encaps, derives the key.
LWE_DEV void st_cluster_u64(uint32_t addr, uint64_t v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// The end of a tree hash on one warp (v: this lane of the root's final
// state, lanes 0..3 the digest): digest mode stores H into out (and out2);
// Encaps mode derives K = H(K' || H(c)) (Alg. 4), one 64-byte block.
LWE_DEV void tree_warp_out(const TreeArgs &a, uint32_t e, const KeccakWarpMap &km, uint32_t lane,
                           uint64_t v) {
  const uint32_t t = lane % 25;
  uint8_t *out;
  if (a.mode == TREE_DIGEST) {
    if (a.out2 && lane < 4) {
      uint8_t *o2 = a.out2 + (size_t)e * a.out2_stride + 8 * lane;
      for (int b = 0; b < 8; b++) o2[b] = (uint8_t)(v >> (8 * b));
    }
    out = a.out + (size_t)e * a.out_stride;
  } else {
    const uint64_t hc = shfl64(v, (lane - 4) & 31);  // lanes 4..7 take the digest
    uint64_t w = 0;
    if (t < 4) w = reinterpret_cast<const uint64_t *>(a.kprime + 32 * (size_t)e)[t];
    else if (t < 8) w = hc;
    if (t == 8) w ^= 0x06;
    if (t == SHA3_RATE / 8 - 1) w ^= 0x8000000000000000ull;
    v = keccak_f1600_warp(km, w);
    out = a.out + 32 * (size_t)e;
  }
  if (lane < 4)
    for (int b = 0; b < 8; b++) out[8 * lane + b] = (uint8_t)(v >> (8 * b));
}

__global__ void __launch_bounds__(TREE_WARP_MAX_THREADS, 1) k_tree_warp(TreeArgs a) {
  extern __shared__ uint64_t sdig[];  // [m][4], used in the cluster's first CTA
  pdl_trigger();
  pdl_wait();
  uint32_t q, nq;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(q));
  asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(nq));
  const uint32_t e = blockIdx.x / nq, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nw = blockDim.x >> 5;
  const KeccakWarpMap km = keccak_warp_map(lane);
  const uint8_t *msg = a.msg_ptrs ? a.msg_ptrs[e] : a.msgs + (size_t)e * a.stride;
  const uint32_t dig0 = cluster_map(sdig, 0);
  for (uint32_t c = q * nw + warp; c < a.m; c += nq * nw) {
    const uint32_t off = c * LWE_TREE_CHUNK;
    const uint64_t v =
        sha3_256_warp_chunk(km, msg + off, min((uint32_t)LWE_TREE_CHUNK, a.len - off), lane);
    if (lane < 4) st_cluster_u64(dig0 + 8 * (4 * c + lane), v);
  }
  cluster_barrier();  // every digest is in the first CTA's shared memory
  if (q != 0 || warp != 0) return;
  tree_warp_out(a, e, km, lane, sha3_256_warp_mem(km, sdig, 32 * a.m, lane));
}

// Tree hash of long messages (more than 32 chunks: ciphertexts and public
// keys of n >= 4096) in two launches.  k_tree_leaves hashes every 1024-byte
// chunk of the batch on its own thread (message e's chunk c on thread
// e m + c, all SMs busy whatever the batch size) and writes the digests to
// a.dig ([count][m][4] words); k_tree_roots then runs each message's root,
// a sequential sponge over 32 m bytes, on one warp with the state spread
// over the lanes, which shortens that chain about twofold against one
// thread (and, for Encaps, derives the key).  k_tree instead gave each such
// message a group of up to 256 threads and ran the root on one thread while
// the group waited.
__global__ void __launch_bounds__(256) k_tree_leaves(TreeArgs a) {
  pdl_trigger();
  pdl_wait();
  const uint64_t L = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= (uint64_t)a.count * a.m) return;
  const uint32_t e = (uint32_t)(L / a.m), c = (uint32_t)(L % a.m);
  const uint8_t *msg = a.msg_ptrs ? a.msg_ptrs[e] : a.msgs + (size_t)e * a.stride;
  const uint32_t off = c * LWE_TREE_CHUNK;
  if (!LWE_BOUNDS(off < a.len && 4 * (L + 1) <= a.dig_words, 114)) return;
  uint64_t s[25];
  sha3_256_global(msg + off, min((uint32_t)LWE_TREE_CHUNK, a.len - off), s);
  uint4 *d = reinterpret_cast<uint4 *>(a.dig + 4 * L);
  d[0] = make_uint4((uint32_t)s[0], (uint32_t)(s[0] >> 32), (uint32_t)s[1], (uint32_t)(s[1] >> 32));
  d[1] = make_uint4((uint32_t)s[2], (uint32_t)(s[2] >> 32), (uint32_t)s[3], (uint32_t)(s[3] >> 32));
}

__global__ void __launch_bounds__(64) k_tree_roots(TreeArgs a) {
  pdl_trigger();
  pdl_wait();
  const uint32_t e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (e >= a.count) return;  // the whole warp
  const KeccakWarpMap km = keccak_warp_map(lane);
  if (!LWE_BOUNDS(4ull * (e + 1) * a.m <= a.dig_words, 115)) return;
  tree_warp_out(a, e, km, lane, sha3_256_warp_mem(km, a.dig + 4ull * e * a.m, 32 * a.m, lane));
}

__global__ void __launch_bounds__(128) k_final_key(FinalKeyArgs a) {
  pdl_trigger();
  pdl_wait();
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
// The 64 x 64 tile sits in shared memory with its 16-byte chunks swizzled:
// chunk q of row r at position q ^ ((r >> 3) & 7).  The transposed read
// (each lane a column, lanes over rows 8 apart) then meets 8 different
// chunks, all 32 banks, where an unswizzled (even a padded) row layout put
// those rows on one or two banks.
LWE_DEV uint32_t limb_tile_at(uint32_t r, uint32_t c) {
  return r * 64 + 8 * ((c >> 3) ^ ((r >> 3) & 7)) + (c & 7);
}

// One instance per source of A: the stored one carries no AES state, so it
// needs few registers and more CTAs per SM keep more loads in flight.
template <bool FUSED>
__global__ void __launch_bounds__(256) k_limbs(GemmLimbArgs a) {
  extern __shared__ uint32_t sT[];
  __shared__ __align__(16) uint16_t tile[64 * 64];
  constexpr bool fused = FUSED;
  const uint32_t n = a.n, ncols = n + (a.B ? 8u : 0u);
  const uint32_t i0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const uint32_t mq = (1u << a.logq) - 1u, mm = mq | (mq << 16);
  AesTab tab;
  uint32_t rk[44];
  pdl_trigger();
  if (fused) {
    aes_fill_smem(sT, g_aes_img);
    __syncthreads();
  }
  pdl_wait();
  if (fused) {
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
    *reinterpret_cast<uint4 *>(&tile[limb_tile_at(r, 8 * cq)]) = v;
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
        const int x = tile[limb_tile_at(8 * ic + t + u, cl)];
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
  pdl_trigger();
  pdl_wait();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    __nv_bfloat16 b = __float2bfloat16_rn((float)S[i]);
    out[i] = *reinterpret_cast<uint16_t *>(&b);
  }
}

#include "pp_kernels.cuh"

// ---------------------------------------------------------------------------
// Host-side launch wrappers (called from lwe_api.cu)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Measurement probes: the instruction sequences of the two integer-bound
// kernels without memory traffic, for their practical peak on this GPU.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_probe_keccak(uint32_t iters, uint32_t *sink) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t s[25];
#pragma unroll
  for (int i = 0; i < 25; i++) s[i] = ((uint64_t)gid << 32) ^ (uint64_t)(i * 0x9E3779B9u);
  for (uint32_t it = 0; it < iters; it++) keccak_f1600(s);
  sink[gid] = (uint32_t)(s[0] ^ s[7] ^ s[24]);
}

__global__ void __launch_bounds__(512, 1) k_probe_aes(uint32_t iters, uint32_t *sink) {
  extern __shared__ uint32_t sT[];
  aes_fill_smem(sT, g_aes_img);
  __syncthreads();
  const AesTab tab = aes_tab(sT);
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t key[4] = {gid, gid * 0x9E3779B9u, ~gid, gid ^ 0x5A5A5A5Au}, rk[44];
  aes_key_expand(tab, key, rk);
  uint32_t acc = 0;
  const uint64_t base = (uint64_t)gid * iters;
  for (uint32_t b = 0; b < iters; b += 2) {  // two blocks in flight, the plain sequence
    const uint4 v = aes_ctr_block(tab, rk, 3, base + b);
    const uint4 w = aes_ctr_block(tab, rk, 3, base + b + 1);
    acc ^= v.x ^ v.y ^ v.z ^ v.w ^ w.x ^ w.y ^ w.z ^ w.w;
  }
  sink[gid] = acc;
}

// The windowed sequence of k_noise: per lane, NOISE_RUN / 32 blocks of one
// run, two at a time; the window constants of 32 runs worked out at once
// (one per lane) and passed by shuffles.
__global__ void __launch_bounds__(512, 1) k_probe_aes_run(uint32_t iters, uint32_t *sink) {
  extern __shared__ uint32_t sT[];
  aes_fill_smem(sT, g_aes_img);
  __syncthreads();
  const AesTab tab = aes_tab(sT);
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
  // one key per warp, as for a run of the noise (the shared window
  // constants depend on it)
  const uint32_t wid = gid >> 5;
  uint32_t key[4] = {wid, wid * 0x9E3779B9u, ~wid, wid ^ 0x5A5A5A5Au}, rk[44];
  aes_key_expand(tab, key, rk);
  uint32_t acc = 0;
  const uint64_t base = (uint64_t)wid * iters * 32;
  constexpr uint32_t PER = NOISE_RUN / 32;  // blocks per lane and run
  for (uint32_t g = 0; g < iters; g += 32 * PER) {
    const AesCtrRun mine = aes_ctr_run(tab, rk, 3, base + 32 * (uint64_t)(g + PER * lane));
    for (uint32_t jr = 0; jr < 32 && g + PER * jr < iters; jr++) {
      const uint64_t first = base + 32 * (uint64_t)(g + PER * jr);
      const AesCtrRun win = aes_ctr_run_shfl(mine, jr);
      const uint32_t x0 = (uint32_t)(first & 255u) + lane;
#pragma unroll
      for (uint32_t j = 0; j < PER; j += 2) {
        const uint4 v = aes_ctr_run_block(tab, rk, win, x0 + 32 * j);
        const uint4 w = aes_ctr_run_block(tab, rk, win, x0 + 32 * j + 32);
        acc ^= v.x ^ v.y ^ v.z ^ v.w ^ w.x ^ w.y ^ w.z ^ w.w;
      }
    }
  }
  sink[gid] = acc;
}

__global__ void __launch_bounds__(32) k_probe_keccak_warp(uint32_t iters, uint32_t *sink) {
  const uint32_t lane = threadIdx.x, t = lane % 25;
  const KeccakWarpMap km = keccak_warp_map(lane);
  uint64_t v = ((uint64_t)blockIdx.x << 32) ^ (uint64_t)(t * 0x9E3779B9u);
  for (uint32_t it = 0; it < iters; it++) v = keccak_f1600_warp(km, v);
  sink[32 * blockIdx.x + lane] = (uint32_t)(v ^ (v >> 32));
}

int launch_probe(int kind, uint32_t ctas, uint32_t iters, uint32_t *sink, cudaStream_t st) {
  if (kind == 0) {
    k_probe_keccak<<<ctas, 256, 0, st>>>(iters, sink);
    return 0;
  }
  if (kind == 1) {
    k_probe_aes<<<ctas, 512, AES_SMEM_BYTES, st>>>(iters, sink);
    return 0;
  }
  if (kind == 2) {
    k_probe_keccak_warp<<<ctas, 32, 0, st>>>(iters, sink);
    return 0;
  }
  if (kind == 3) {
    k_probe_aes_run<<<ctas, 512, AES_SMEM_BYTES, st>>>(iters, sink);
    return 0;
  }
  return -1;
}

static int grid_for(uint64_t work, int per_cta, int max_ctas) {
  uint64_t g = (work + per_cta - 1) / per_cta;
  if (g > (uint64_t)max_ctas) g = max_ctas;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t lwe_upload_aes_table(const uint32_t T0[256]) {
  cudaError_t e = cudaMemcpyToSymbol(g_aes_T0, T0, 256 * sizeof(uint32_t));
  if (e != cudaSuccess) return e;
  std::vector<uint32_t> img(AES_TABLE_WORDS);
  for (uint32_t i = 0; i < AES_TABLE_WORDS; i++) img[i] = aes_table_word(T0, i);
  return cudaMemcpyToSymbol(g_aes_img, img.data(), AES_TABLE_WORDS * sizeof(uint32_t));
}

cudaError_t lwe_kernel_smem_setup() {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_expand_A, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_noise, cudaFuncAttributeMaxDynamicSharedMemorySize, NOISE_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_noise_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           NOISE_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_mul_as_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int fused_smem = AES_SMEM_BYTES + SA_PAIRS * 16 + 2048 * 4;
  e = cudaFuncSetAttribute(k_sa_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fused_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sa_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fused_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_probe_aes, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_probe_aes_run, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pp_expand_A, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pp_noise, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_limbs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, AES_SMEM_BYTES);
  return e;
}

void launch_expand_A(const uint8_t *seeds, uint32_t seed_stride, uint32_t count, uint32_t n,
                     uint32_t logq, uint16_t *A, uint64_t a_stride, int num_sms, cudaStream_t st) {
  const uint64_t nblk = (uint64_t)n * n / 8;
  const int gx = grid_for(nblk, 512 * 4, num_sms);
  launch_k(k_expand_A, dim3(gx, count), 512, AES_SMEM_BYTES, st, seeds, seed_stride, n, logq, A,
           a_stride);
}

void launch_noise_table(const NoiseArgs &a, int8_t *out, cudaStream_t st) {
  launch_k(k_noise_table, 1, 512, NOISE_SMEM_BYTES, st, a, out);
}

void launch_noise(const NoiseArgs &a, int num_sms, cudaStream_t st) {
  const int g = grid_for((uint64_t)a.count * a.runs_per_item, 16, num_sms);
  launch_k(k_noise, g, 512, NOISE_SMEM_BYTES, st, a);
}

void launch_mul_as(const MulAsArgs &a, uint32_t count, bool fused, int num_sms, cudaStream_t st) {
  const uint32_t rows = a.rows ? a.rows : a.n;
  if (fused) {
    const uint32_t per_item = std::max<uint32_t>(1u, (uint32_t)std::max(num_sms, 1) / count);
    dim3 grid(std::min((rows + 15) / 16, per_item), count);
    launch_k(k_mul_as_fused, grid, 512, AES_SMEM_BYTES, st, a);
  } else if ((uint64_t)count * (rows / AS_ROWS) < 4ull * 16 * (uint64_t)std::max(num_sms, 1)) {
    // fewer than ~4 row groups per warp of the grid below: split columns
    launch_k(k_mul_as_split, dim3(rows / AS_ROWS, count), 256, 0, st, a);
  } else {
    // two CTAs per SM in all, spread over the items
    const uint32_t want = (rows / AS_ROWS + 7) / 8;
    const uint32_t share = std::max<uint32_t>(1u, 2u * (uint32_t)std::max(num_sms, 1) / count);
    dim3 grid(std::min(want, share), count);
    launch_k(k_mul_as_rows, grid, 256, 0, st, a);
  }
}

void launch_decrypt(const DecryptArgs &a, uint32_t count, cudaStream_t st) {
  launch_k(k_decrypt, count, 256, 0, st, a);
}

void launch_mul_sa(const MulSaArgs &a, uint32_t items, bool fused, bool cmp, int num_sms,
                   cudaStream_t st) {
  // rows split over a cluster of R CTAs (R a power of two <= 8) until the
  // grid holds about two CTAs per SM (one with the AES tables)
  const uint32_t cbs = (a.n + 255) / 256;
  const uint32_t target = (fused ? 1u : 2u) * (uint32_t)std::max(num_sms, 1);
  const uint32_t pairs = ((a.row1 ? a.row1 : a.n) - a.row0) / 2;
  uint32_t R = 1;
  while (R < 8 && (uint64_t)cbs * items * R < target && pairs / (2 * R) >= 64) R <<= 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cbs, R, items);
  cfg.dynamicSmemBytes = (fused ? AES_SMEM_BYTES : 0) + SA_PAIRS * 16 + 2048 * 4;
  cfg.blockDim = dim3(fused ? 512 : 256, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = g_launch_pdl ? 1 : 0;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = 1;
  attr[1].val.clusterDim.y = R;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = R > 1 ? 2 : 1;
  if (fused) {
    if (cmp)
      cudaLaunchKernelEx(&cfg, k_sa_fused<true>, a);
    else
      cudaLaunchKernelEx(&cfg, k_sa_fused<false>, a);
  } else {
    if (cmp)
      cudaLaunchKernelEx(&cfg, k_sa<true>, a);
    else
      cudaLaunchKernelEx(&cfg, k_sa<false>, a);
  }
}

void launch_v_encode(const VEncArgs &a, uint32_t count, bool cmp, cudaStream_t st) {
  if (cmp)
    launch_k(k_v_encode<true>, count, 256, 0, st, a);
  else
    launch_k(k_v_encode<false>, count, 256, 0, st, a);
}

void launch_keygen_seeds(const KeygenSeedArgs &a, uint32_t warp_max, cudaStream_t st) {
  if (a.count <= warp_max) {
    launch_k(k_keygen_seeds_warp, a.count, 96, 0, st, a);
    return;
  }
  launch_k(k_keygen_seeds, (a.count + 63) / 64, 64, 0, st, a);
}

void launch_derive(const DeriveArgs &a, uint32_t warp_max, cudaStream_t st) {
  if (a.count <= warp_max) {
    launch_k(k_derive_warp, a.count, 64, 0, st, a);
    return;
  }
  launch_k(k_derive, (a.count + 31) / 32, 64, 0, st, a);
}

// One CTA per SM where the batch allows (the leaf work is one wave: CTAs of
// equal size spread it evenly), at most TREE_MAX_THREADS threads and 48 KB
// of digests per CTA.
void launch_tree(TreeArgs &a, int num_sms, uint32_t warp_max, cudaStream_t st) {
  a.m = (a.len + LWE_TREE_CHUNK - 1) / LWE_TREE_CHUNK;
  if (a.count <= warp_max) {
    // about four warps per SM: chunks over a cluster of up to 8 CTAs
    const uint32_t q = std::max<uint32_t>(1, std::min<uint32_t>(8, (a.m + 3) / 4));
    const uint32_t w = std::min<uint32_t>((a.m + q - 1) / q, TREE_WARP_MAX_THREADS / 32);
    launch_k_cluster(k_tree_warp, a.count * q, 32 * w, (size_t)a.m * 32, st, q, a);
    return;
  }
  const uint32_t sms = num_sms > 0 ? (uint32_t)num_sms : 1u;
  if (a.m > 32 && a.dig && (uint64_t)a.count * a.m * 4 <= a.dig_words) {
    // long messages: every leaf on its own thread, then one warp per root,
    // once k_tree (below: one thread per message runs its root) would have
    // root chains of more than 128 chunks (31+ sequential permutations) or
    // need more than one wave of two CTAs per SM
    uint32_t t = 1;
    while (t < a.m && t < 256) t <<= 1;
    const uint32_t cap = std::max<uint32_t>(
        1u, std::min<uint32_t>(TREE_MAX_THREADS / t, (48u * 1024u) / (8u * (4 * a.m + 1))));
    if (a.m > 128 || a.count > 2 * sms * cap) {
      // small leaf CTAs when the batch fills the SMs only a few warps deep
      const uint64_t leaves = (uint64_t)a.count * a.m;
      const uint32_t lt = leaves >= (uint64_t)sms * 1024 ? 256u : 64u;
      launch_k(k_tree_leaves, (uint32_t)((leaves + lt - 1) / lt), lt, 0, st, a);
      launch_k(k_tree_roots, (a.count + 1) / 2, 64, 0, st, a);
      return;
    }
  }
  {
    // the balanced schedule of k_tree_bal: leaves of full length filling
    // more than 12 and at most 13 warps per CTA, every message's short
    // chunk and root on one warp
    const uint32_t last = a.len - (a.m - 1) * LWE_TREE_CHUNK;
    const uint32_t ml = a.m - (last < LWE_TREE_CHUNK ? 1u : 0u);
    const uint32_t ipc = (a.count + sms - 1) / sms;
    const uint32_t nl = ipc * ml;
    const size_t smem = ((size_t)ipc * (4 * a.m + 1) + 25 * TB_SLOTS) * 8;
    if (a.m >= 2 && nl > 12 * 32 && nl <= 13 * 32 && ipc <= 32 && smem <= 48 * 1024 &&
        (a.count + ipc - 1) / ipc <= sms) {
      a.ipc = ipc;
      a.ml = ml;
      launch_k(k_tree_bal, (a.count + ipc - 1) / ipc, 512, smem, st, a);
      return;
    }
    // leaves of at most 12 warps: dense packing, roots on the least loaded
    // SMSP (warp 12 + s of SMSP s)
    const size_t smem_d = (size_t)ipc * (4 * a.m + 1) * 8;
    if (a.m >= 2 && ml >= 1 && nl <= 12 * 32 && ipc <= 32 && smem_d <= 48 * 1024 &&
        (a.count + ipc - 1) / ipc <= sms) {
      const uint32_t wl = (nl + 31) / 32;
      uint32_t best = 3, load_best = 99;
      for (int sp = 3; sp >= 0; sp--) {
        const uint32_t load = wl > (uint32_t)sp ? (wl - 1 - sp) / 4 + 1 : 0;  // leaf warps on SMSP sp
        if (load < load_best) {
          load_best = load;
          best = (uint32_t)sp;
        }
      }
      a.ipc = ipc;
      a.ml = ml;
      a.rw = 12 + best;
      launch_k(k_tree_dense, (a.count + ipc - 1) / ipc, 512, smem_d, st, a);
      return;
    }
  }
  uint32_t t = 1;
  while (t < a.m && t < 256) t <<= 1;
  a.tpi = t;
  const uint32_t words = 4 * a.m + 1;
  uint32_t cap = TREE_MAX_THREADS / t;
  cap = std::min<uint32_t>(cap, (48u * 1024u) / (8u * words));
  cap = std::max<uint32_t>(cap, 1u);
  a.ipc = std::min<uint32_t>(cap, (a.count + sms - 1) / sms);
  if (a.ipc == 0) a.ipc = 1;
  const uint32_t threads = (a.ipc * t + 31) / 32 * 32;
  const size_t smem = (size_t)a.ipc * words * 8;
  launch_k(k_tree, (a.count + a.ipc - 1) / a.ipc, threads, smem, st, a);
}

void launch_final_key(const FinalKeyArgs &a, uint32_t warp_max, cudaStream_t st) {
  if (a.count <= warp_max) {
    launch_k(k_final_key_warp, a.count, 32, 0, st, a);
    return;
  }
  launch_k(k_final_key, (a.count + 127) / 128, 128, 0, st, a);
}

void launch_gemm_limbs(const GemmLimbArgs &a, int num_sms, cudaStream_t st) {
  (void)num_sms;
  const uint32_t ncols = a.n + (a.B ? 8u : 0u);
  dim3 grid((ncols + 63) / 64, (a.n + 63) / 64);
  if (a.A)
    launch_k(k_limbs<false>, grid, 256, 0, st, a);
  else
    launch_k(k_limbs<true>, grid, 256, AES_SMEM_BYTES, st, a);
}

void launch_s_to_bf16(const int8_t *S, uint64_t count, uint16_t *out, int num_sms, cudaStream_t st) {
  const int g = grid_for(count, 256 * 8, num_sms * 8);
  launch_k(k_s_to_bf16, g, 256, 0, st, S, count, out);
}

// ---- the paper's own parameter profile ------------------------------------
void launch_pp_expand_A(const uint8_t *seedA, uint32_t n, ModQ M, uint32_t *A, int num_sms,
                        cudaStream_t st) {
  const int g = grid_for((uint64_t)n * n / 4, 512 * 4, num_sms);
  launch_k(k_pp_expand_A, g, 512, AES_SMEM_BYTES, st, seedA, n, M, A);
}

void launch_pp_noise(const PpNoiseArgs &a, int num_sms, cudaStream_t st) {
  uint64_t blocks = 0;
  for (uint32_t s = 0; s < a.nout; s++)
    blocks += a.o[s].kind == PP_BINOMIAL ? (a.o[s].count + 15) / 16 : (a.o[s].count + 7) / 8;
  launch_k(k_pp_noise, grid_for(blocks, 512 * 4, num_sms), 512, AES_SMEM_BYTES, st, a);
}

void launch_pp_as(const PpAsArgs &a, cudaStream_t st) {
  launch_k(k_pp_as, (a.n + 7) / 8, 256, 0, st, a);
}

void launch_pp_encrypt(const PpEncArgs &a, bool cmp, cudaStream_t st) {
  const dim3 grid(a.n / PPE_BN, PP_MBITS / PPE_BM);
  if (cmp)
    launch_k(k_pp_encrypt<true>, grid, 256, 0, st, a);
  else
    launch_k(k_pp_encrypt<false>, grid, 256, 0, st, a);
}

void launch_pp_v(const PpVArgs &a, bool cmp, cudaStream_t st) {
  if (cmp)
    launch_k(k_pp_v<true>, PP_MBITS, 256, 0, st, a);
  else
    launch_k(k_pp_v<false>, PP_MBITS, 256, 0, st, a);
}

void launch_pp_decrypt(const PpDecArgs &a, cudaStream_t st) {
  launch_k(k_pp_decrypt, PP_MBITS, 256, 0, st, a);
}

void launch_pp_limbs(const uint32_t *A, uint32_t n, uint32_t q, uint16_t *limbs, cudaStream_t st) {
  launch_k(k_pp_limbs, dim3(n / 64, n / 64), 256, 0, st, A, n, q, limbs);
}
