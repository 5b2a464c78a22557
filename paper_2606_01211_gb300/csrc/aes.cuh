// aes.cuh -- warp-parallel AES-128 in counter mode for sm_103a.
//
// The public matrix A and all noise are expanded on the device from short
// seeds (device-resident random number generation, Sec. 3.3 of the paper),
// here with AES-128 (FIPS-197) in counter mode: the keystream block for
// (domain d, index b) is AES_k(BE64(d) || BE64(b)).
//
// Implementation: the round-table formulation of AES (SubBytes + ShiftRows +
// MixColumns folded into four 256-word tables T0..T3, Tk = T0 rotated left
// by 8k), state held little-endian in four registers.  The tables live in
// shared memory, each replicated 32 times so that lane l only ever reads
// bank l (conflict-free).  The layout is chosen so that ONE byte-permute
// instruction forms a lookup address: entry x of table k for lane l sits at
//     (k >> 1) * 65536 + x * 256 + (k & 1) * 128 + 4 l   bytes,
// and prmt(state, 4 l) with the state byte placed in byte 1 yields
// x * 256 + 4 l; the table is selected by the instruction's immediate offset.
// This keeps the integer ALU pipe (half the lane rate of the FMA pipe on
// this part) to one permute per lookup plus the XORs.  The last round and the
// key schedule read S(x) from the table whose byte in the needed position
// holds S(x) (T0 holds S in bytes 1 and 2).
#pragma once
#include "common.cuh"

// T0[x] = 2.S(x) | S(x) << 8 | S(x) << 16 | 3.S(x) << 24, filled by the host.
#define AES_TABLE_WORDS (2 * 16384)
#define AES_SMEM_BYTES (AES_TABLE_WORDS * 4)  // 128 KB

// The tables in this layout, word i: table k = 2 (i >> 14) + ((i >> 5) & 1),
// entry (i >> 6) & 255.  The host builds the whole 128 KB image once per
// device (aes_table_image); a CTA copies it into shared memory with 16-byte
// loads instead of working out every word.
inline uint32_t aes_table_word(const uint32_t T0[256], uint32_t i) {
  const uint32_t k = 2 * (i >> 14) + ((i >> 5) & 1);
  const uint32_t v = T0[(i >> 6) & 255];
  return k ? (v << (8 * k)) | (v >> (32 - 8 * k)) : v;
}

LWE_DEV void aes_fill_smem(uint32_t *sT, const uint4 *img) {
  uint4 *d = reinterpret_cast<uint4 *>(sT);
#pragma unroll 4
  for (int i = threadIdx.x; i < AES_TABLE_WORDS / 4; i += blockDim.x) d[i] = img[i];
}

struct AesTab {
  const char *base;  // shared-memory tables
  uint32_t lane4;    // 4 * lane in byte 0

  // entry T_K[byte BYTE of s] for this lane
  template <int K, int BYTE>
  LWE_DEV uint32_t T(uint32_t s) const {
    const uint32_t off = __byte_perm(s, lane4, 0x5504 | (BYTE << 4));
    return *reinterpret_cast<const uint32_t *>(base + off + (K >> 1) * 65536 + (K & 1) * 128);
  }
};

LWE_DEV AesTab aes_tab(const uint32_t *sT) {
  AesTab t;
  t.base = reinterpret_cast<const char *>(sT);
  t.lane4 = (threadIdx.x & 31) << 2;
  return t;
}

// SubWord(RotWord(w)) for a little-endian word: output byte r is S(byte
// r+1 of w), read from the table holding S at byte r (T3, T0, T1, T2).
LWE_DEV uint32_t aes_subrot(const AesTab &tab, uint32_t w) {
  return (tab.T<3, 1>(w) & 0x000000ffu) | (tab.T<0, 2>(w) & 0x0000ff00u) |
         (tab.T<1, 3>(w) & 0x00ff0000u) | (tab.T<2, 0>(w) & 0xff000000u);
}

// FIPS-197 5.2 key expansion on little-endian words; Rcon enters byte 0 and
// stays in GF(2^8).
LWE_DEV void aes_key_expand(const AesTab &tab, const uint32_t key[4], uint32_t rk[44]) {
  rk[0] = key[0];
  rk[1] = key[1];
  rk[2] = key[2];
  rk[3] = key[3];
  uint32_t rcon = 1;
#pragma unroll
  for (int i = 4; i < 44; i++) {
    uint32_t t = rk[i - 1];
    if ((i & 3) == 0) {
      t = aes_subrot(tab, t) ^ rcon;
      rcon = ((rcon << 1) ^ ((rcon & 0x80u) ? 0x1bu : 0u)) & 0xffu;
    }
    rk[i] = rk[i - 4] ^ t;
  }
}

// One AES-128 encryption of the little-endian state (s0..s3).  New column c
// takes row k from old column c + k (ShiftRows); the row-k contribution is
// T_k (MixColumns).
LWE_DEV void aes_encrypt(const AesTab &tab, const uint32_t rk[44], uint32_t &s0, uint32_t &s1,
                         uint32_t &s2, uint32_t &s3) {
  s0 ^= rk[0];
  s1 ^= rk[1];
  s2 ^= rk[2];
  s3 ^= rk[3];
#pragma unroll
  for (int r = 1; r < 10; r++) {
    const uint32_t t0 = tab.T<0, 0>(s0) ^ tab.T<1, 1>(s1) ^ tab.T<2, 2>(s2) ^ tab.T<3, 3>(s3) ^ rk[4 * r + 0];
    const uint32_t t1 = tab.T<0, 0>(s1) ^ tab.T<1, 1>(s2) ^ tab.T<2, 2>(s3) ^ tab.T<3, 3>(s0) ^ rk[4 * r + 1];
    const uint32_t t2 = tab.T<0, 0>(s2) ^ tab.T<1, 1>(s3) ^ tab.T<2, 2>(s0) ^ tab.T<3, 3>(s1) ^ rk[4 * r + 2];
    const uint32_t t3 = tab.T<0, 0>(s3) ^ tab.T<1, 1>(s0) ^ tab.T<2, 2>(s1) ^ tab.T<3, 3>(s2) ^ rk[4 * r + 3];
    s0 = t0;
    s1 = t1;
    s2 = t2;
    s3 = t3;
  }
  // final round: SubBytes + ShiftRows + AddRoundKey; output byte r of a
  // column is S(x), read from the table with S at byte r
  const uint32_t o0 = (tab.T<3, 0>(s0) & 0x000000ffu) | (tab.T<0, 1>(s1) & 0x0000ff00u) |
                      (tab.T<1, 2>(s2) & 0x00ff0000u) | (tab.T<2, 3>(s3) & 0xff000000u);
  const uint32_t o1 = (tab.T<3, 0>(s1) & 0x000000ffu) | (tab.T<0, 1>(s2) & 0x0000ff00u) |
                      (tab.T<1, 2>(s3) & 0x00ff0000u) | (tab.T<2, 3>(s0) & 0xff000000u);
  const uint32_t o2 = (tab.T<3, 0>(s2) & 0x000000ffu) | (tab.T<0, 1>(s3) & 0x0000ff00u) |
                      (tab.T<1, 2>(s0) & 0x00ff0000u) | (tab.T<2, 3>(s1) & 0xff000000u);
  const uint32_t o3 = (tab.T<3, 0>(s3) & 0x000000ffu) | (tab.T<0, 1>(s0) & 0x0000ff00u) |
                      (tab.T<1, 2>(s1) & 0x00ff0000u) | (tab.T<2, 3>(s2) & 0xff000000u);
  s0 = o0 ^ rk[40];
  s1 = o1 ^ rk[41];
  s2 = o2 ^ rk[42];
  s3 = o3 ^ rk[43];
}

// Keystream block (domain, index) as four little-endian words: the sixteen
// output bytes in order, i.e. eight little-endian 16-bit words.
LWE_DEV uint4 aes_ctr_block(const AesTab &tab, const uint32_t rk[44], uint64_t domain,
                            uint64_t index) {
  uint32_t s0 = bswap32((uint32_t)(domain >> 32));
  uint32_t s1 = bswap32((uint32_t)domain);
  uint32_t s2 = bswap32((uint32_t)(index >> 32));
  uint32_t s3 = bswap32((uint32_t)index);
  aes_encrypt(tab, rk, s0, s1, s2, s3);
  return make_uint4(s0, s1, s2, s3);
}

// Counter blocks that differ only in the low byte of the index.  Inside a
// 256-aligned window of indices the input block varies in its last byte
// alone, which is byte 3 of s3.  After ShiftRows that byte feeds one column
// of round 1 (t0, through T3), and t0 feeds one lookup of each column of
// round 2.  So 15 of round 1's 16 lookups and 12 of round 2's are the same
// for the whole window: AesCtrRun holds their XORs (with the round keys),
// and a block of the window costs 1 + 4 + 8 x 16 = 133 lookups instead of
// 160.  The result is the same AES-128 encryption, bit for bit.
struct AesCtrRun {
  uint32_t s3;      // s3 ^ rk[3] of the window's first index (low byte 0)
  uint32_t k0;      // round 1, column 0 without the varying lookup
  uint32_t k1, k2, k3, k4;  // round 2, columns 0..3 without the varying lookup
};

// Window of `index` (its low byte ignored) in stream `domain`.
LWE_DEV AesCtrRun aes_ctr_run(const AesTab &tab, const uint32_t rk[44], uint64_t domain,
                              uint64_t index) {
  const uint32_t s0 = bswap32((uint32_t)(domain >> 32)) ^ rk[0];
  const uint32_t s1 = bswap32((uint32_t)domain) ^ rk[1];
  const uint32_t s2 = bswap32((uint32_t)(index >> 32)) ^ rk[2];
  const uint32_t s3 = bswap32((uint32_t)index & ~0xffu) ^ rk[3];
  AesCtrRun w;
  w.s3 = s3;
  w.k0 = tab.T<0, 0>(s0) ^ tab.T<1, 1>(s1) ^ tab.T<2, 2>(s2) ^ rk[4];
  const uint32_t t1 = tab.T<0, 0>(s1) ^ tab.T<1, 1>(s2) ^ tab.T<2, 2>(s3) ^ tab.T<3, 3>(s0) ^ rk[5];
  const uint32_t t2 = tab.T<0, 0>(s2) ^ tab.T<1, 1>(s3) ^ tab.T<2, 2>(s0) ^ tab.T<3, 3>(s1) ^ rk[6];
  const uint32_t t3 = tab.T<0, 0>(s3) ^ tab.T<1, 1>(s0) ^ tab.T<2, 2>(s1) ^ tab.T<3, 3>(s2) ^ rk[7];
  w.k1 = tab.T<1, 1>(t1) ^ tab.T<2, 2>(t2) ^ tab.T<3, 3>(t3) ^ rk[8];
  w.k2 = tab.T<0, 0>(t1) ^ tab.T<1, 1>(t2) ^ tab.T<2, 2>(t3) ^ rk[9];
  w.k3 = tab.T<0, 0>(t2) ^ tab.T<1, 1>(t3) ^ tab.T<3, 3>(t1) ^ rk[10];
  w.k4 = tab.T<0, 0>(t3) ^ tab.T<2, 2>(t1) ^ tab.T<3, 3>(t2) ^ rk[11];
  return w;
}

// The window constants held by lane `src`, for the whole warp (every lane
// calls it): a warp works out 32 windows at once, one per lane, and takes
// them one after another.
LWE_DEV AesCtrRun aes_ctr_run_shfl(const AesCtrRun &w, uint32_t src) {
  AesCtrRun o;
  o.s3 = __shfl_sync(0xffffffffu, w.s3, src);
  o.k0 = __shfl_sync(0xffffffffu, w.k0, src);
  o.k1 = __shfl_sync(0xffffffffu, w.k1, src);
  o.k2 = __shfl_sync(0xffffffffu, w.k2, src);
  o.k3 = __shfl_sync(0xffffffffu, w.k3, src);
  o.k4 = __shfl_sync(0xffffffffu, w.k4, src);
  return o;
}

// Keystream block of index (window base | x), x < 256; equal to
// aes_ctr_block for that index.
LWE_DEV uint4 aes_ctr_run_block(const AesTab &tab, const uint32_t rk[44], const AesCtrRun &w,
                                uint32_t x) {
  const uint32_t t0 = w.k0 ^ tab.T<3, 3>(w.s3 ^ (x << 24));
  uint32_t s0 = tab.T<0, 0>(t0) ^ w.k1;
  uint32_t s1 = tab.T<3, 3>(t0) ^ w.k2;
  uint32_t s2 = tab.T<2, 2>(t0) ^ w.k3;
  uint32_t s3 = tab.T<1, 1>(t0) ^ w.k4;
#pragma unroll
  for (int r = 3; r < 10; r++) {
    const uint32_t t0 = tab.T<0, 0>(s0) ^ tab.T<1, 1>(s1) ^ tab.T<2, 2>(s2) ^ tab.T<3, 3>(s3) ^ rk[4 * r + 0];
    const uint32_t t1 = tab.T<0, 0>(s1) ^ tab.T<1, 1>(s2) ^ tab.T<2, 2>(s3) ^ tab.T<3, 3>(s0) ^ rk[4 * r + 1];
    const uint32_t t2 = tab.T<0, 0>(s2) ^ tab.T<1, 1>(s3) ^ tab.T<2, 2>(s0) ^ tab.T<3, 3>(s1) ^ rk[4 * r + 2];
    const uint32_t t3 = tab.T<0, 0>(s3) ^ tab.T<1, 1>(s0) ^ tab.T<2, 2>(s1) ^ tab.T<3, 3>(s2) ^ rk[4 * r + 3];
    s0 = t0;
    s1 = t1;
    s2 = t2;
    s3 = t3;
  }
  const uint32_t o0 = (tab.T<3, 0>(s0) & 0x000000ffu) | (tab.T<0, 1>(s1) & 0x0000ff00u) |
                      (tab.T<1, 2>(s2) & 0x00ff0000u) | (tab.T<2, 3>(s3) & 0xff000000u);
  const uint32_t o1 = (tab.T<3, 0>(s1) & 0x000000ffu) | (tab.T<0, 1>(s2) & 0x0000ff00u) |
                      (tab.T<1, 2>(s3) & 0x00ff0000u) | (tab.T<2, 3>(s0) & 0xff000000u);
  const uint32_t o2 = (tab.T<3, 0>(s2) & 0x000000ffu) | (tab.T<0, 1>(s3) & 0x0000ff00u) |
                      (tab.T<1, 2>(s0) & 0x00ff0000u) | (tab.T<2, 3>(s1) & 0xff000000u);
  const uint32_t o3 = (tab.T<3, 0>(s3) & 0x000000ffu) | (tab.T<0, 1>(s0) & 0x0000ff00u) |
                      (tab.T<1, 2>(s1) & 0x00ff0000u) | (tab.T<2, 3>(s2) & 0xff000000u);
  return make_uint4(o0 ^ rk[40], o1 ^ rk[41], o2 ^ rk[42], o3 ^ rk[43]);
}

// Load a 16-byte key from memory as four little-endian words.
LWE_DEV void aes_load_key(const uint8_t *key, uint32_t k[4]) {
  if ((reinterpret_cast<uintptr_t>(key) & 15) == 0) {
    uint4 v = *reinterpret_cast<const uint4 *>(key);
    k[0] = v.x;
    k[1] = v.y;
    k[2] = v.z;
    k[3] = v.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; i++)
      k[i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) |
             ((uint32_t)key[4 * i + 2] << 16) | ((uint32_t)key[4 * i + 3] << 24);
  }
}

// Key expansion from a plain 256-word T0 table (global memory, or a copy in
// shared memory), for kernels that do not hold the rotated shared tables
// (one key per thread, off the hot loop).
LWE_DEV void aes_key_expand_global(const uint32_t *T0g, const uint32_t key[4], uint32_t rk[44]) {
  rk[0] = key[0];
  rk[1] = key[1];
  rk[2] = key[2];
  rk[3] = key[3];
  uint32_t rcon = 1;
#pragma unroll
  for (int i = 4; i < 44; i++) {
    uint32_t t = rk[i - 1];
    if ((i & 3) == 0) {
      t = __funnelshift_r(t, t, 8);
      t = ((T0g[t & 0xff] >> 8) & 0xffu) | (T0g[(t >> 8) & 0xff] & 0xff00u) |
          (T0g[(t >> 16) & 0xff] & 0xff0000u) | ((T0g[t >> 24] << 16) & 0xff000000u);
      t ^= rcon;
      rcon = ((rcon << 1) ^ ((rcon & 0x80u) ? 0x1bu : 0u)) & 0xffu;
    }
    rk[i] = rk[i - 4] ^ t;
  }
}
