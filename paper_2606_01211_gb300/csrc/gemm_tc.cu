// gemm_tc.cu -- exact mod-2^D product S' [A | B] on the sm_103a tensor cores.
//
// Batching many encryptions against one public key stacks their S' (Alg. 2)
// into one tall matrix, so that B' = S' A + E' and V = S' B + E'' become one
// dense contraction with K = n.  sm_103a has no integer tcgen05 MMA, so the
// product is made exact on the bf16 path:
//
//   A[i][c] = lo + 256 hi (mod 2^16),  lo, hi in [-128, 127] (bf16-exact)
//   S'[r][i] in [-c, c]                                       (bf16-exact)
//   P_lo = S' lo,  P_hi = S' hi accumulate in fp32; every partial sum is an
//   integer of magnitude <= n c 128 < 2^24, so fp32 holds it exactly.
//   out = (P_lo + 256 P_hi + E) mod 2^D
//
// Kernel shape: persistent, one 128 x BN output tile at a time per CTA,
// warp-specialised: warp 0 issues TMA loads of S' and limb tiles (128B
// swizzle) into a 4-stage shared-memory ring, warp 1 issues tcgen05.mma
// (M = 128, N = 2 BN: the lo and hi limb tiles side by side, K = 16) into one
// of two TMEM accumulators, warps 2-5 drain the other accumulator with
// tcgen05.ld, fold the limbs, add the noise (and the encoded message for the
// C columns) and store -- or compare against a received ciphertext (Decaps).
// Every mbarrier wait is bounded; a wait that runs out raises the context's
// device error word and the CTA leaves cleanly.
//
// k_gemm_sa2 is the same product on CTA pairs (a cluster of two CTAs on one
// TPC, tcgen05 cta_group::2): one tile is 256 rows x 128 columns; each CTA
// loads its own 128 rows of S' and ONE limb tile (rank 0 the lo limbs, rank
// 1 the hi limbs), and the leader's MMA (M = 256, N = 256) reads the B
// operand from both CTAs' shared memory.  Per SM and k-block that is 32 KB
// of operands instead of 48 KB for the same 128 x 256 products.  Both
// CTAs' copies complete on the leader's full barrier; the leader's commits
// are multicast to both CTAs' empty / accumulator-full barriers; each
// epilogue warp of either CTA signals the leader's accumulator-empty
// barrier.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "gemm_tc.h"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // bf16 elements = 128 bytes = one swizzle atom row
constexpr int STAGES = 4;
constexpr int NTHREADS = 192;
constexpr uint64_t kTimeoutNs = 1000000000ull;  // 1 s per wait
constexpr uint64_t kDrainNs = 2000000ull;       // 2 ms for copies in flight after an abort

template <int BN>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 2;          // 16 KB
  static constexpr int B_BYTES = 2 * BN * BK * 2;      // lo + hi tiles
  static constexpr int STAGE_TX = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = 2 * (2 * BN);       // two accumulators
  static constexpr int BAR_OFF = STAGES * (A_BYTES + B_BYTES);
  static constexpr int SMEM = BAR_OFF + 256 + 1024;    // + barriers + align
  // instruction descriptor, kind::f16: D f32, A/B bf16, K-major, N = 2 BN,
  // M = 128
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(2 * BN / 8) << 17) |
                                    ((uint32_t)(BM / 16) << 24);
};

// CTA-pair variant: per CTA 128 rows of S' and one limb tile of BN2
// columns per stage; MMA M = 256 (the pair), N = 2 BN2 (lo | hi).
constexpr int BN2 = 128;
constexpr int STAGES2 = 6;
constexpr int NTHREADS2 = 64 + 8 * 32;  // producer, MMA, 8 epilogue warps
struct Cfg2 {
  static constexpr int A_BYTES = BM * BK * 2;        // 16 KB
  static constexpr int B_BYTES = BN2 * BK * 2;       // 16 KB: one limb
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = 2 * (2 * BN2);    // two accumulators
  static constexpr int BAR_OFF = STAGES2 * STAGE_BYTES;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(2 * BN2 / 8) << 17) |
                                    ((uint32_t)(2 * BM / 16) << 24);
};

LWE_DEV uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

LWE_DEV uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

LWE_DEV void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

LWE_DEV void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

LWE_DEV void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

LWE_DEV bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false when another role gave up or the limit ran out.
LWE_DEV bool wait_bar(uint32_t bar, uint32_t parity, volatile uint32_t *abort_flag,
                      uint32_t *dev_err, uint64_t limit_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicOr(dev_err, LWE_DEVERR_TIMEOUT);
      return false;
    }
  }
}

// The same decision for every lane of a warp (the epilogue's TMEM loads and
// shuffles are warp-collective, so no lane may leave the loop alone).
LWE_DEV bool wait_bar_warp(uint32_t bar, uint32_t parity, volatile uint32_t *abort_flag,
                           uint32_t *dev_err) {
  const bool ok = wait_bar(bar, parity, abort_flag, dev_err);
  return __all_sync(0xffffffffu, ok);
}

LWE_DEV void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

LWE_DEV void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// The same copies for a CTA pair: the mbarrier may live in the peer CTA
// (a shared::cluster address).
LWE_DEV void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

LWE_DEV void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

LWE_DEV uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared::cluster address of this CTA's shared variable `a` in CTA `rank`
LWE_DEV uint32_t peer_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

LWE_DEV void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

LWE_DEV void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

LWE_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
LWE_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05 format): K-major, 128-byte
// swizzle, 8-row core groups 1024 bytes apart (stride byte offset), version
// bits 46-48 = 0b001, swizzle mode 2 (128B) in bits 61-63.
LWE_DEV uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

LWE_DEV void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                      uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

LWE_DEV void mma_bf16_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on the barrier at this offset in every CTA of `mask` once the
// pair's earlier MMAs have completed
LWE_DEV void mma_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

LWE_DEV void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

LWE_DEV void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

LWE_DEV void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

LWE_DEV uint32_t fold(uint32_t lo_bits, uint32_t hi_bits) {
  const int lo = __float2int_rn(__uint_as_float(lo_bits));
  const int hi = __float2int_rn(__uint_as_float(hi_bits));
  return (uint32_t)lo + ((uint32_t)hi << 8);
}

// The same fold for |lo|, |hi| < 2^22: x + 1.5 * 2^23 is exact and its bit
// pattern is 0x4B400000 + x, whose low 16 bits are x mod 2^16, so two
// FP32 adds replace the two float-to-integer conversions.
LWE_DEV uint32_t fold_small(uint32_t lo_bits, uint32_t hi_bits) {
  const uint32_t lo = __float_as_uint(__fadd_rn(__uint_as_float(lo_bits), 12582912.0f));
  const uint32_t hi = __float_as_uint(__fadd_rn(__uint_as_float(hi_bits), 12582912.0f));
  return lo + (hi << 8);
}

// The global operands of CHUNKS 16-column chunks of this thread's row from
// column n0 (zero where absent): E' and, for Decaps (ov != nullptr), the
// received B'.  Issued ahead of the accumulator wait so that the load
// latency overlaps the tile's MMAs.
template <int CHUNKS, bool ODDQ = false>
LWE_DEV void epilogue_prefetch(const GemmSaArgs &a, uint32_t row, uint32_t n0, uint4 *ev,
                               uint4 *ov) {
  if (ODDQ) ov = nullptr;  // the odd-modulus epilogue reads the received rows itself
  const bool rv = row < a.rows;
  const uint8_t *obase = a.out + (size_t)(row >> 3) * a.out_stride + 2 * (size_t)(row & 7) * a.n;
#pragma unroll
  for (int cc = 0; cc < CHUNKS; cc++) {
    const uint32_t c = n0 + 16 * cc;
    const bool in = rv && c < a.n;
    ev[cc] = make_uint4(0, 0, 0, 0);
    if (a.E && in) ev[cc] = __ldg(reinterpret_cast<const uint4 *>(a.E + (size_t)row * a.n + c));
    if (ov) {
      ov[2 * cc] = make_uint4(0, 0, 0, 0);
      ov[2 * cc + 1] = ov[2 * cc];
      if (a.cmp && in) {
        const uint4 *o = reinterpret_cast<const uint4 *>(obase + 2 * (size_t)c);
        ov[2 * cc] = __ldg(o);
        ov[2 * cc + 1] = __ldg(o + 1);
      }
    }
  }
}

// x mod q for x < 2^32 (Barrett: m = floor(2^32 / q); one correction)
LWE_DEV uint32_t oq_mod(uint32_t x, uint32_t q, uint32_t m) {
  const uint32_t r = x - __umulhi(x, m) * q;
  return r >= q ? r - q : r;
}

LWE_DEV uint32_t oq_mod_s(int32_t x, uint32_t q, uint32_t m) {  // |x| < 2^31
  const uint32_t r = oq_mod((uint32_t)(x < 0 ? -x : x), q, m);
  return (x < 0 && r) ? q - r : r;
}

// The odd-modulus epilogue (paper profile): the limbs' exact FP32 sums lo,
// hi give (lo + 256 hi) mod q; add the K-split running sum (uint32 mod q)
// and, in the final pass, E1 (int8), then store the row's uint32 entries or
// compare them with the received ciphertext (item = row / 256).
template <int CHUNKS>
LWE_DEV void epilogue_tile_oddq(const GemmSaArgs &a, uint32_t row, uint32_t n0, uint32_t tl,
                                uint32_t hi_off, const uint4 *ev) {
  const uint32_t q = a.oddq_q, m = a.oddq_m;
  const bool rv = row < a.rows;
  uint32_t *orow = reinterpret_cast<uint32_t *>(a.out) + (size_t)row * a.n;
  uint32_t diff = 0;
#pragma unroll
  for (uint32_t cc = 0; cc < CHUNKS; cc++) {
    const uint32_t c = n0 + 16 * cc;
    uint32_t lo[16], hi[16];
    tmem_ld16(tl + 16 * cc, lo);
    tmem_ld16(tl + hi_off + 16 * cc, hi);
    tmem_wait_ld();
    if (rv && c < a.ncols) {
      uint32_t v[16];
#pragma unroll
      for (int t = 0; t < 16; t++) {
        const int l = __float2int_rn(__uint_as_float(lo[t]));
        const int h = __float2int_rn(__uint_as_float(hi[t]));
        v[t] = oq_mod(oq_mod_s(l, q, m) + oq_mod(256u * oq_mod_s(h, q, m), q, m), q, m);
      }
      if (a.partial_in) {
        const uint4 *pin = reinterpret_cast<const uint4 *>(
            reinterpret_cast<const uint32_t *>(a.partial_in) + (size_t)row * a.ncols + c);
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const uint4 p = __ldg(pin + u);
          v[4 * u] = oq_mod(v[4 * u] + p.x, q, m);
          v[4 * u + 1] = oq_mod(v[4 * u + 1] + p.y, q, m);
          v[4 * u + 2] = oq_mod(v[4 * u + 2] + p.z, q, m);
          v[4 * u + 3] = oq_mod(v[4 * u + 3] + p.w, q, m);
        }
      }
      uint4 *dst;
      if (a.partial_out) {
        dst = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(a.partial_out) +
                                        (size_t)row * a.ncols + c);
      } else {
        if (a.E) {
          const uint32_t ew[4] = {ev[cc].x, ev[cc].y, ev[cc].z, ev[cc].w};
#pragma unroll
          for (int t = 0; t < 16; t++) v[t] = oq_mod(v[t] + oq_mod_s(sext8(ew[t >> 2], t & 3), q, m), q, m);
        }
        dst = reinterpret_cast<uint4 *>(orow + c);
        if (a.cmp) {
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const uint4 g = __ldg(dst + u);
            diff |= (g.x ^ v[4 * u]) | (g.y ^ v[4 * u + 1]) | (g.z ^ v[4 * u + 2]) |
                    (g.w ^ v[4 * u + 3]);
          }
          continue;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u++)
        dst[u] = make_uint4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
    }
  }
  if (a.cmp && !a.partial_out) {
    diff = __reduce_or_sync(0xffffffffu, diff);
    if (rv && (row & 31) == 0 && diff) atomicOr(a.flags + (row >> 8), 1u);
  }
}

// CHUNKS 16-column chunks of one output row of this CTA from its TMEM
// accumulator (lo limb products at column tl + j, hi at tl + hi_off + j):
// fold the limbs, add the K-split running sum, E' (B' columns) or E'' +
// Enc(mu) (C columns), then store, or compare with the received ciphertext
// and flag a mismatch.  `row` is this thread's output row, n0 the first
// column, tl the TMEM address of the first lo column of its lane quarter.
// The received B' comes from ov when given (prefetched with the E'), else
// it is loaded here one chunk ahead of its use.
template <int CHUNKS, bool ODDQ = false>
LWE_DEV void epilogue_tile(const GemmSaArgs &a, uint32_t row, uint32_t n0, uint32_t tl,
                           uint32_t hi_off, const uint4 *ev, const uint4 *ov) {
  if (ODDQ) {
    epilogue_tile_oddq<CHUNKS>(a, row, n0, tl, hi_off, ev);
    return;
  }
  const uint32_t D = a.logq, mask = (1u << D) - 1u;
  const bool rv = row < a.rows;
  const uint32_t e = row >> 3, kk = row & 7;
  uint8_t *obase = a.out + (size_t)e * a.out_stride;
  uint32_t diff = 0;
  uint4 o_cur0 = make_uint4(0, 0, 0, 0), o_cur1 = o_cur0;
  auto fetch = [&](uint32_t cc, uint4 &o0, uint4 &o1) {
    const uint32_t c = n0 + 16 * cc;
    if (a.cmp && rv && c < a.n) {
      const uint4 *o = reinterpret_cast<const uint4 *>(obase + 2 * ((size_t)kk * a.n + c));
      o0 = __ldg(o);
      o1 = __ldg(o + 1);
    }
  };
  if (!ov) fetch(0, o_cur0, o_cur1);
#pragma unroll
  for (uint32_t cc = 0; cc < CHUNKS; cc++) {
    const uint32_t c = n0 + 16 * cc;
    uint32_t lo[16], hi[16];
    tmem_ld16(tl + 16 * cc, lo);
    tmem_ld16(tl + hi_off + 16 * cc, hi);
    uint4 o_nxt0 = make_uint4(0, 0, 0, 0), o_nxt1 = o_nxt0;
    if (ov) {
      o_cur0 = ov[2 * cc];
      o_cur1 = ov[2 * cc + 1];
    } else if (cc + 1 < CHUNKS) {
      fetch(cc + 1, o_nxt0, o_nxt1);
    }
    tmem_wait_ld();
    if (rv && c < a.ncols) {
      uint32_t v[16];
      if (a.fast_fold) {
#pragma unroll
        for (int t = 0; t < 16; t++) v[t] = fold_small(lo[t], hi[t]);
      } else {
#pragma unroll
        for (int t = 0; t < 16; t++) v[t] = fold(lo[t], hi[t]);
      }
      const uint32_t nvalid = min(16u, a.ncols - c);
      if (a.partial_in) {  // running sum of the earlier K passes
        const uint16_t *pin = a.partial_in + (size_t)row * a.ncols + c;
        if (nvalid == 16) {
          const uint4 p0 = __ldg(reinterpret_cast<const uint4 *>(pin));
          const uint4 p1 = __ldg(reinterpret_cast<const uint4 *>(pin) + 1);
          const uint32_t pw[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
          for (int t = 0; t < 16; t++) v[t] += (pw[t >> 1] >> (16 * (t & 1))) & 0xffffu;
        } else {  // ragged last columns; unrolled so that v stays in registers
#pragma unroll
          for (uint32_t t = 0; t < 16; t++)
            if (t < nvalid) v[t] += pin[t];
        }
      }
      if (a.partial_out) {  // non-final pass: keep the running sum
        uint16_t *pout = a.partial_out + (size_t)row * a.ncols + c;
        if (nvalid == 16) {
          uint32_t w[8];
#pragma unroll
          for (int t = 0; t < 8; t++) w[t] = (v[2 * t] & 0xffffu) | (v[2 * t + 1] << 16);
          reinterpret_cast<uint4 *>(pout)[0] = make_uint4(w[0], w[1], w[2], w[3]);
          reinterpret_cast<uint4 *>(pout)[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
#pragma unroll
          for (uint32_t t = 0; t < 16; t++)
            if (t < nvalid) pout[t] = (uint16_t)v[t];
        }
      } else if (c < a.n) {  // B' columns: 16 at once (n is a multiple of 16)
        if (a.E) {
          const uint32_t ew[4] = {ev[cc].x, ev[cc].y, ev[cc].z, ev[cc].w};
#pragma unroll
          for (int t = 0; t < 16; t++) v[t] += (uint32_t)sext8(ew[t >> 2], t & 3);
        }
        uint32_t w[8];
#pragma unroll
        for (int t = 0; t < 8; t++) w[t] = (v[2 * t] & mask) | ((v[2 * t + 1] & mask) << 16);
        if (a.cmp) {
          diff |= (o_cur0.x ^ w[0]) | (o_cur0.y ^ w[1]) | (o_cur0.z ^ w[2]) |
                  (o_cur0.w ^ w[3]) | (o_cur1.x ^ w[4]) | (o_cur1.y ^ w[5]) |
                  (o_cur1.z ^ w[6]) | (o_cur1.w ^ w[7]);
        } else if (LWE_BOUNDS(row < a.rows && c + 16 <= a.n, 202)) {
          uint4 *o = reinterpret_cast<uint4 *>(obase + 2 * ((size_t)kk * a.n + c));
          o[0] = make_uint4(w[0], w[1], w[2], w[3]);
          o[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
      } else {  // V columns n..n+7: C = V + E'' + Enc(mu)
        const uint32_t Bb = a.B;
        const uint8_t *mu = a.mu + 32 * (size_t)e + kk * Bb;
        uint32_t bits = 0;
        for (uint32_t t = 0; t < Bb; t++) bits |= (uint32_t)mu[t] << (8 * t);
        const int8_t *epp = a.Epp + 64 * (size_t)e + 8 * kk;
        uint16_t *co = reinterpret_cast<uint16_t *>(obase + 16 * (size_t)a.n) + 8 * kk;
#pragma unroll
        for (int t = 0; t < 8; t++) {
          const uint32_t sym = (bits >> (t * Bb)) & ((1u << Bb) - 1u);
          const uint32_t cv = (v[t] + (uint32_t)(int)epp[t] + (sym << (D - Bb))) & mask;
          if (a.cmp)
            diff |= cv ^ (uint32_t)co[t];
          else
            co[t] = (uint16_t)cv;
        }
      }
    }
    if (!ov) {
      o_cur0 = o_nxt0;
      o_cur1 = o_nxt1;
    }
  }
  if (a.cmp) {
    diff |= __shfl_xor_sync(0xffffffffu, diff, 1);
    diff |= __shfl_xor_sync(0xffffffffu, diff, 2);
    diff |= __shfl_xor_sync(0xffffffffu, diff, 4);
    if (rv && kk == 0 && diff) atomicOr(a.flags + e, 1u);
  }
}

// Tile order.  Tiles are visited in groups of g M-blocks (g = a.group_m):
// inside a group the M-block varies fastest, so the tiles that the
// persistent CTAs hold at one time share g row slabs of S' and about
// (CTAs / g) limb slabs of [A | B].  With g = 1 this is the row-major order
// (all column tiles of one M-block, then the next), which suits an [A | B]
// that stays in L2; for a large n (limb slabs of several MB per pass) it
// would re-stream every limb slab from HBM once per M-block.
LWE_DEV void tile_mn(uint32_t tile, uint32_t num_m, uint32_t num_n, uint32_t g, uint32_t &tm,
                     uint32_t &tn) {
  if (g <= 1) {
    tm = tile / num_n;
    tn = tile - tm * num_n;
    return;
  }
  const uint32_t per = g * num_n;
  const uint32_t m_first = (tile / per) * g, idx = tile % per;
  const uint32_t gm = min(g, num_m - m_first);
  tm = m_first + idx % gm;
  tn = idx / gm;
}

template <int BN, bool ODDQ>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm_sa(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmL,
              const GemmSaArgs a) {
  using C = Cfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::BAR_OFF);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], done
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
  volatile uint32_t *abort_flag = tmem_slot + 1;

  pdl_trigger();
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t num_m = (a.rows + BM - 1) / BM;
  const uint32_t num_n = (a.ncols + BN - 1) / BN;
  const uint32_t num_tiles = num_m * num_n;
  const uint32_t KB = a.kblocks;

  auto bar = [&](int i) { return smem_u32(bars + i); };
  auto full = [&](uint32_t s) { return bar(s); };
  auto empty = [&](uint32_t s) { return bar(STAGES + s); };
  auto tfull = [&](uint32_t x) { return bar(2 * STAGES + x); };
  auto tempty = [&](uint32_t x) { return bar(2 * STAGES + 2 + x); };
  const uint32_t done_bar = bar(2 * STAGES + 4);
  auto sA = [&](uint32_t s) { return smem_u32(smem + s * C::A_BYTES); };
  auto sB = [&](uint32_t s) { return smem_u32(smem + STAGES * C::A_BYTES + s * C::B_BYTES); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int x = 0; x < 2; x++) {
      mbar_init(tfull(x), 1);
      mbar_init(tempty(x), 4 * 32);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmS)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmL)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();  // the operands are written by the previous kernels of the stream

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    uint32_t stage = 0, phase = 0;
    uint32_t issued = 0;  // bit s: stage s has a load in flight or done
    uint32_t last_phase = 0;  // bit s: phase of stage s's last load
    bool ok = true;
    for (uint32_t tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x) {
      uint32_t tm, tn;
      tile_mn(tile, num_m, num_n, a.group_m, tm, tn);
      const int m0 = (int)(tm * BM);
      const int n0 = (int)(tn * BN);
      for (uint32_t kb = 0; kb < KB; kb++) {
        if (!wait_bar(empty(stage), phase ^ 1, abort_flag, a.dev_err)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(full(stage), C::STAGE_TX);
        tma_load_2d(sA(stage), &tmS, (int)(a.k0 + kb * BK), m0, full(stage));
        tma_load_3d(sB(stage), &tmL, (int)(a.k0 + kb * BK), n0, 0, full(stage));
        issued |= 1u << stage;
        last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    if (!ok) {
      // let every copy already issued land before the CTA leaves
      for (uint32_t s = 0; s < STAGES; s++) {
        if (!(issued & (1u << s))) continue;
        const uint32_t ph = (last_phase >> s) & 1u;
        const uint64_t t0 = gtime();
        while (!mbar_try_wait(full(s), ph) && gtime() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    uint32_t stage = 0, phase = 0, it = 0;
    bool ok = true;
    for (uint32_t tile = blockIdx.x; ok && tile < num_tiles; tile += gridDim.x, ++it) {
      const uint32_t acc = it & 1, use = it >> 1;
      if (!wait_bar(tempty(acc), (use & 1) ^ 1, abort_flag, a.dev_err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem_base + acc * (2 * BN);
      for (uint32_t kb = 0; kb < KB; kb++) {
        if (!wait_bar(full(stage), phase, abort_flag, a.dev_err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = sdesc(sA(stage)), bd = sdesc(sB(stage));
#pragma unroll
        for (uint32_t kk = 0; kk < BK / 16; kk++)
          mma_bf16(d, ad + 2 * kk, bd + 2 * kk, C::IDESC, (kb | kk) != 0);
        mma_commit(empty(stage));
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (ok) mma_commit(tfull(acc));
    }
    // all issued MMAs complete before TMEM is released
    mma_commit(done_bar);
    const uint64_t t0 = gtime();
    while (!mbar_try_wait(done_bar, 0) && gtime() - t0 < kTimeoutNs) {
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const uint32_t q = warp & 3;  // TMEM lane quarter of this warp
    uint32_t it = 0;
    for (uint32_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++it) {
      const uint32_t acc = it & 1, use = it >> 1;
      uint32_t tm, tn;
      tile_mn(tile, num_m, num_n, a.group_m, tm, tn);
      const uint32_t m0 = tm * BM, n0 = tn * BN;
      const uint32_t row = m0 + 32 * q + lane;
      uint4 ev[BN / 16];
      epilogue_prefetch<BN / 16, ODDQ>(a, row, n0, ev, nullptr);
      if (!wait_bar_warp(tfull(acc), use & 1, abort_flag, a.dev_err)) break;
      tc_fence_after();
      epilogue_tile<BN / 16, ODDQ>(a, row, n0, tmem_base + ((32 * q) << 16) + acc * (2 * BN), BN,
                                   ev, nullptr);
      tc_fence_before();
      mbar_arrive(tempty(acc));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
}

// CTA-pair kernel (see the file head).  Roles per CTA as in k_gemm_sa;
// only the leader (rank 0) issues MMAs.  Tiles: 256 rows (rank r owns rows
// 128 r .. 128 r + 127 of the tile) x BN2 columns, both CTAs of a cluster
// walking the same tile sequence.
template <bool ODDQ>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS2, 1)
    k_gemm_sa2(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmL,
               const GemmSaArgs a) {
  using C = Cfg2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::BAR_OFF);
  // bars: full[STAGES2] (leader), empty[STAGES2], tfull[2], tempty[2]
  // (leader), done (leader)
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES2 + 5);
  volatile uint32_t *abort_flag = tmem_slot + 1;

  pdl_trigger();
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
  const uint32_t num_m = (a.rows + 2 * BM - 1) / (2 * BM);
  const uint32_t num_n = (a.ncols + BN2 - 1) / BN2;
  const uint32_t num_tiles = num_m * num_n;
  const uint32_t KB = a.kblocks;

  auto bar = [&](int i) { return smem_u32(bars + i); };
  auto full = [&](uint32_t s) { return bar(s); };
  auto empty = [&](uint32_t s) { return bar(STAGES2 + s); };
  auto tfull = [&](uint32_t x) { return bar(2 * STAGES2 + x); };
  auto tempty = [&](uint32_t x) { return bar(2 * STAGES2 + 2 + x); };
  const uint32_t done_bar = bar(2 * STAGES2 + 4);
  auto sA = [&](uint32_t s) { return smem_u32(smem + s * C::STAGE_BYTES); };
  auto sB = [&](uint32_t s) { return smem_u32(smem + s * C::STAGE_BYTES + C::A_BYTES); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES2; s++) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int x = 0; x < 2; x++) {
      mbar_init(tfull(x), 1);
      mbar_init(tempty(x), 2 * 8);  // one arrival per epilogue warp of each CTA
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmS)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmL)) : "memory");
  }
  if (warp == 1) {  // one warp of each CTA of the pair allocates together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // the peer's barriers exist before any copy or arrive targets them
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();  // the operands are written by the previous kernels of the stream

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    uint32_t stage = 0, phase = 0;
    uint32_t armed = 0, last_phase = 0;  // leader: stages with a phase in flight
    bool ok = true;
    for (uint32_t tile = cluster; ok && tile < num_tiles; tile += nclusters) {
      uint32_t tm, tn;
      tile_mn(tile, num_m, num_n, a.group_m, tm, tn);
      const int m0 = (int)(tm * 2 * BM + rank * BM);
      const int n0 = (int)(tn * BN2);
      // a tail tile whose second half has no rows: the peer loads no S'
      // (its accumulator rows are never stored) but still its limb tile
      const bool peer_rows = tm * 2 * BM + BM < a.rows;
      const uint32_t tx = 2 * C::STAGE_BYTES - (peer_rows ? 0u : (uint32_t)C::A_BYTES);
      for (uint32_t kb = 0; kb < KB; kb++) {
        if (!wait_bar(empty(stage), phase ^ 1, abort_flag, a.dev_err)) {
          ok = false;
          break;
        }
        const uint32_t fb = peer_addr(full(stage), 0);
        if (leader) {
          mbar_arrive_expect_tx(full(stage), tx);
          armed |= 1u << stage;
          last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
        }
        if (leader || peer_rows) tma_load_2d_pair(sA(stage), &tmS, (int)(a.k0 + kb * BK), m0, fb);
        tma_load_3d_pair(sB(stage), &tmL, (int)(a.k0 + kb * BK), n0, (int)rank, fb);
        if (++stage == STAGES2) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    if (!ok) {
      // let the copies already issued land before the CTA leaves: the
      // leader sees both CTAs' bytes on its full barriers; the peer cannot
      // observe its own copies and waits out the drain time
      const uint64_t t0 = gtime();
      if (leader) {
        for (uint32_t s = 0; s < STAGES2; s++) {
          if (!(armed & (1u << s))) continue;
          const uint32_t ph = (last_phase >> s) & 1u;
          while (!mbar_try_wait(full(s), ph) && gtime() - t0 < kDrainNs) {
          }
        }
      }
      while (gtime() - t0 < kDrainNs) {
      }
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (leader only) ----------------
    uint32_t stage = 0, phase = 0, it = 0;
    bool ok = true;
    for (uint32_t tile = cluster; ok && tile < num_tiles; tile += nclusters, ++it) {
      const uint32_t acc = it & 1, use = it >> 1;
      if (!wait_bar(tempty(acc), (use & 1) ^ 1, abort_flag, a.dev_err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem_base + acc * (2 * BN2);
      for (uint32_t kb = 0; kb < KB; kb++) {
        if (!wait_bar(full(stage), phase, abort_flag, a.dev_err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = sdesc(sA(stage)), bd = sdesc(sB(stage));
#pragma unroll
        for (uint32_t kk = 0; kk < BK / 16; kk++)
          mma_bf16_pair(d, ad + 2 * kk, bd + 2 * kk, C::IDESC, (kb | kk) != 0);
        mma_commit_pair(empty(stage), 0x3);
        if (++stage == STAGES2) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (ok) mma_commit_pair(tfull(acc), 0x3);
    }
    // all issued MMAs complete before either CTA releases TMEM or leaves
    mma_commit_pair(done_bar, 0x1);
    const uint64_t t0 = gtime();
    while (!mbar_try_wait(done_bar, 0) && gtime() - t0 < kTimeoutNs) {
    }
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs) ----------------
    const uint32_t q = warp & 3;  // TMEM lane quarter of this warp
    const uint32_t half = (warp - 2) >> 2;  // which 64 of the tile's 128 columns
    // this thread's row and first column in tile t, worked out once per
    // tile (before its accumulator is ready) and kept for its drain
    uint32_t row = 0, col = 0;
    auto coords = [&](uint32_t t) {
      uint32_t tm, tn;
      tile_mn(t, num_m, num_n, a.group_m, tm, tn);
      row = tm * 2 * BM + rank * BM + 32 * q + lane;
      col = tn * BN2 + half * (BN2 / 2);
    };
    // the next tile's E' / received B' are loaded while this tile drains
    uint4 ev[BN2 / 32], ov[BN2 / 16];
    uint32_t it = 0;
    if (cluster < num_tiles) {
      coords(cluster);
      epilogue_prefetch<BN2 / 32, ODDQ>(a, row, col, ev, ov);
    }
    for (uint32_t tile = cluster; tile < num_tiles; tile += nclusters, ++it) {
      const uint32_t acc = it & 1, use = it >> 1;
      if (!wait_bar_warp(tfull(acc), use & 1, abort_flag, a.dev_err)) break;
      tc_fence_after();
      epilogue_tile<BN2 / 32, ODDQ>(a, row, col,
                              tmem_base + ((32 * q) << 16) + acc * (2 * BN2) + half * (BN2 / 2),
                              BN2, ev, ov);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(peer_addr(tempty(acc), 0));
      const uint32_t next = tile + nclusters;
      if (next < num_tiles) {
        coords(next);
        epilogue_prefetch<BN2 / 32, ODDQ>(a, row, col, ev, ov);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // no MMA, copy or arrive of the pair is left when either CTA frees TMEM
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
}

// Exercises the bounded wait of the pipeline on a barrier that no thread
// and no copy ever completes: the wait must give up after limit_ns, raise
// the device error word and let the kernel finish.  Nothing faults.
__global__ void k_selftest_wait(uint32_t *dev_err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ uint32_t abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) wait_bar(smem_u32(&bar), 0, &abort_flag, dev_err, limit_ns);
  __syncthreads();
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

LWE_BOUNDS_READER(lwe_bounds_read_gemm)

namespace {

bool make_map(CUtensorMap *m, const void *base, int rank, const cuuint64_t *dims,
              const cuuint64_t *strides, const cuuint32_t *box) {
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void *>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN>
int launch_bn(const GemmSaArgs &a, int num_sms, cudaStream_t st) {
  using C = Cfg<BN>;
  CUtensorMap tmS, tmL;
  const cuuint64_t dS[2] = {a.n, a.rows};
  const cuuint64_t sS[1] = {2ull * a.n};
  const cuuint32_t bS[2] = {BK, BM};
  const cuuint64_t dL[3] = {a.n, a.ncols, 2};
  const cuuint64_t sL[2] = {2ull * a.n, 2ull * a.n * a.ncols};
  const cuuint32_t bL[3] = {BK, BN, 2};
  if (!make_map(&tmS, a.S, 2, dS, sS, bS)) return LWE_ECUDA;
  if (!make_map(&tmL, a.limbs, 3, dL, sL, bL)) return LWE_ECUDA;
  const uint32_t tiles = ((a.rows + BM - 1) / BM) * ((a.ncols + BN - 1) / BN);
  const int grid = (int)(tiles < (uint32_t)num_sms ? tiles : (uint32_t)num_sms);
  if (a.oddq_q)
    launch_k(k_gemm_sa<BN, true>, grid, NTHREADS, C::SMEM, st, tmS, tmL, a);
  else
    launch_k(k_gemm_sa<BN, false>, grid, NTHREADS, C::SMEM, st, tmS, tmL, a);
  return LWE_OK;
}

int launch_pair(const GemmSaArgs &a, int num_sms, cudaStream_t st) {
  CUtensorMap tmS, tmL;
  const cuuint64_t dS[2] = {a.n, a.rows};
  const cuuint64_t sS[1] = {2ull * a.n};
  const cuuint32_t bS[2] = {BK, BM};
  const cuuint64_t dL[3] = {a.n, a.ncols, 2};
  const cuuint64_t sL[2] = {2ull * a.n, 2ull * a.n * a.ncols};
  const cuuint32_t bL[3] = {BK, BN2, 1};
  if (!make_map(&tmS, a.S, 2, dS, sS, bS)) return LWE_ECUDA;
  if (!make_map(&tmL, a.limbs, 3, dL, sL, bL)) return LWE_ECUDA;
  const uint32_t tiles = ((a.rows + 2 * BM - 1) / (2 * BM)) * ((a.ncols + BN2 - 1) / BN2);
  const uint32_t pairs = (uint32_t)(num_sms / 2);
  const uint32_t clusters = tiles < pairs ? tiles : pairs;
  if (a.oddq_q)
    launch_k(k_gemm_sa2<true>, 2 * clusters, NTHREADS2, Cfg2::SMEM, st, tmS, tmL, a);
  else
    launch_k(k_gemm_sa2<false>, 2 * clusters, NTHREADS2, Cfg2::SMEM, st, tmS, tmL, a);
  return LWE_OK;
}

}  // namespace

cudaError_t lwe_gemm_setup() {
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cudaError_t e = cudaSuccess;
  for (auto k : {k_gemm_sa<128, false>, k_gemm_sa<128, true>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<128>::SMEM);
    if (e != cudaSuccess) return e;
  }
  for (auto k : {k_gemm_sa<64, false>, k_gemm_sa<64, true>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<64>::SMEM);
    if (e != cudaSuccess) return e;
  }
  for (auto k : {k_gemm_sa2<false>, k_gemm_sa2<true>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg2::SMEM);
    if (e != cudaSuccess) return e;
  }
  return e;
}

// The fp32 accumulator is exact while every partial sum stays below 2^24:
// K * c * 128 < 2^24 for the K contracted in one pass.
uint32_t lwe_gemm_kchunk(uint32_t clip) {
  const uint32_t k = ((1u << 24) - 1u) / (clip * 128u);
  return k / BK * BK;
}

uint32_t lwe_gemm_passes(uint32_t n, uint32_t clip) {
  const uint32_t kc = lwe_gemm_kchunk(clip);
  return (n + kc - 1) / kc;
}

bool lwe_gemm_supported(uint32_t n, uint32_t logq, uint32_t clip) {
  (void)logq;
  return n >= 64 && clip >= 1 && lwe_gemm_kchunk(clip) >= BK;
}

// One launch per K pass; the running sum lives in a.partial_out between them.
int launch_gemm_sa(const GemmSaArgs &a, int num_sms, cudaStream_t st) {
  if (!g_encode) return LWE_ECUDA;
  if (a.rows == 0) return LWE_OK;
  const uint32_t kmax = a.kchunk ? a.kchunk : a.n;
  const uint32_t np = (a.n + kmax - 1) / kmax;
  // passes of equal K (multiples of BK, none above kmax): a short last pass
  // would be all epilogue (n = 32768 at kmax 10880: 8192 x 4 instead of
  // 10880 x 3 + 128)
  const uint32_t kc = np > 1 ? ((a.n + np - 1) / np + BK - 1) / BK * BK : kmax;
  const uint32_t passes = (a.n + kc - 1) / kc;
  if (passes > 1 && !a.partial_out) return LWE_EINVAL;
  for (uint32_t p = 0; p < passes; p++) {
    GemmSaArgs b = a;
    b.k0 = p * kc;
    b.kblocks = (min(a.n, b.k0 + kc) - b.k0 + BK - 1) / BK;
    b.partial_in = p > 0 ? a.partial_out : nullptr;
    b.partial_out = p + 1 < passes ? a.partial_out : nullptr;
    // |partial sums| <= K c 128 (zero-filled K tail included)
    b.fast_fold = (uint64_t)b.kblocks * BK * a.clip * 128u < (1u << 22) ? 1 : 0;
    // tile order: group the row blocks once this pass's limbs (2 limbs x 2
    // bytes x ncols x K) outgrow a quarter of L2
    if (!b.group_m)
      b.group_m = 4ull * a.ncols * (uint64_t)b.kblocks * BK > (32ull << 20) ? 8u : 1u;
    const int rc = a.pair && num_sms >= 2 ? launch_pair(b, num_sms, st)
                   : a.bn == 64           ? launch_bn<64>(b, num_sms, st)
                                          : launch_bn<128>(b, num_sms, st);
    if (rc != LWE_OK) return rc;
  }
  return LWE_OK;
}

void launch_selftest_wait(uint32_t *dev_err, uint64_t limit_ns, cudaStream_t st) {
  k_selftest_wait<<<1, 32, 0, st>>>(dev_err, limit_ns);
}
