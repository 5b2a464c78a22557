// aes.cuh -- warp-parallel AES-128 in counter mode for sm_103a.
//
// The public matrix A and all noise are expanded on the device from short
// seeds (device-resident random number generation, Sec. 3.3 of the paper),
// here with AES-128 (FIPS-197) in counter mode: the keystream block for
// (domain d, index b) is AES_k(BE64(d) || BE64(b)).
//
// Implementation: the 4x32-bit round-table formulation of AES (SubBytes +
// ShiftRows + MixColumns folded into one table T0 of 256 words and its byte
// rotations), with the state held little-endian in four registers.  The table
// lives in shared memory replicated 32 times so that lane l always reads bank
// l: a warp's 32 lookups are one conflict-free wavefront.  The last round
// takes the S-box from the bytes of T0 that hold S(x).
#pragma once
#include "common.cuh"

// T0[x] = 2.S(x) | S(x) << 8 | S(x) << 16 | 3.S(x) << 24  (little-endian
// column contribution of the row-0 byte); filled by the host at start-up.
#define AES_TABLE_WORDS (256 * 32)
#define AES_SMEM_BYTES (AES_TABLE_WORDS * 4)

// Replicate the 256-word table so that entry x for lane l sits at x*32 + l.
LWE_DEV void aes_fill_smem(uint32_t *sT, const uint32_t *T0g) {
  for (int i = threadIdx.x; i < AES_TABLE_WORDS; i += blockDim.x)
    sT[i] = T0g[i >> 5];
}

struct AesTab {
  const uint32_t *lane_base;  // sT + lane
  LWE_DEV uint32_t t0(uint32_t byte) const { return lane_base[byte << 5]; }
  LWE_DEV uint32_t sbox(uint32_t byte) const { return (t0(byte) >> 8) & 0xffu; }
};

LWE_DEV AesTab aes_tab(const uint32_t *sT) {
  AesTab t;
  t.lane_base = sT + (threadIdx.x & 31);
  return t;
}

LWE_DEV uint32_t byte_of(uint32_t w, int k) {
  return __byte_perm(w, 0, 0x4440 | k);
}

// FIPS-197 5.2 key expansion on little-endian words.  RotWord of a
// little-endian word is a right rotation by 8; Rcon enters the low byte.
LWE_DEV void aes_key_expand(const AesTab &tab, const uint32_t key[4],
                            uint32_t rk[44]) {
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
      t = tab.sbox(byte_of(t, 0)) | (tab.sbox(byte_of(t, 1)) << 8) |
          (tab.sbox(byte_of(t, 2)) << 16) | (tab.sbox(byte_of(t, 3)) << 24);
      t ^= rcon;
      rcon = ((rcon << 1) ^ ((rcon & 0x80u) ? 0x1bu : 0u)) & 0xffu;
    }
    rk[i] = rk[i - 4] ^ t;
  }
}

// One AES-128 encryption of the little-endian state (s0..s3).
LWE_DEV void aes_encrypt(const AesTab &tab, const uint32_t rk[44],
                         uint32_t &s0, uint32_t &s1, uint32_t &s2,
                         uint32_t &s3) {
  s0 ^= rk[0];
  s1 ^= rk[1];
  s2 ^= rk[2];
  s3 ^= rk[3];
#pragma unroll
  for (int r = 1; r < 10; r++) {
    // new column c takes row k from old column c + k (ShiftRows); the
    // row-k contribution is T0 rotated left by 8k (MixColumns)
    uint32_t t0 = tab.t0(byte_of(s0, 0)) ^ rotl32(tab.t0(byte_of(s1, 1)), 8) ^
                  rotl32(tab.t0(byte_of(s2, 2)), 16) ^
                  rotl32(tab.t0(byte_of(s3, 3)), 24) ^ rk[4 * r + 0];
    uint32_t t1 = tab.t0(byte_of(s1, 0)) ^ rotl32(tab.t0(byte_of(s2, 1)), 8) ^
                  rotl32(tab.t0(byte_of(s3, 2)), 16) ^
                  rotl32(tab.t0(byte_of(s0, 3)), 24) ^ rk[4 * r + 1];
    uint32_t t2 = tab.t0(byte_of(s2, 0)) ^ rotl32(tab.t0(byte_of(s3, 1)), 8) ^
                  rotl32(tab.t0(byte_of(s0, 2)), 16) ^
                  rotl32(tab.t0(byte_of(s1, 3)), 24) ^ rk[4 * r + 2];
    uint32_t t3 = tab.t0(byte_of(s3, 0)) ^ rotl32(tab.t0(byte_of(s0, 1)), 8) ^
                  rotl32(tab.t0(byte_of(s1, 2)), 16) ^
                  rotl32(tab.t0(byte_of(s2, 3)), 24) ^ rk[4 * r + 3];
    s0 = t0;
    s1 = t1;
    s2 = t2;
    s3 = t3;
  }
  // final round: SubBytes + ShiftRows + AddRoundKey.  S(x) is byte 1 and
  // byte 2 of T0[x].
  uint32_t o0 = ((tab.t0(byte_of(s0, 0)) >> 8) & 0x000000ffu) |
                (tab.t0(byte_of(s1, 1)) & 0x0000ff00u) |
                (tab.t0(byte_of(s2, 2)) & 0x00ff0000u) |
                ((tab.t0(byte_of(s3, 3)) << 16) & 0xff000000u);
  uint32_t o1 = ((tab.t0(byte_of(s1, 0)) >> 8) & 0x000000ffu) |
                (tab.t0(byte_of(s2, 1)) & 0x0000ff00u) |
                (tab.t0(byte_of(s3, 2)) & 0x00ff0000u) |
                ((tab.t0(byte_of(s0, 3)) << 16) & 0xff000000u);
  uint32_t o2 = ((tab.t0(byte_of(s2, 0)) >> 8) & 0x000000ffu) |
                (tab.t0(byte_of(s3, 1)) & 0x0000ff00u) |
                (tab.t0(byte_of(s0, 2)) & 0x00ff0000u) |
                ((tab.t0(byte_of(s1, 3)) << 16) & 0xff000000u);
  uint32_t o3 = ((tab.t0(byte_of(s3, 0)) >> 8) & 0x000000ffu) |
                (tab.t0(byte_of(s0, 1)) & 0x0000ff00u) |
                (tab.t0(byte_of(s1, 2)) & 0x00ff0000u) |
                ((tab.t0(byte_of(s2, 3)) << 16) & 0xff000000u);
  s0 = o0 ^ rk[40];
  s1 = o1 ^ rk[41];
  s2 = o2 ^ rk[42];
  s3 = o3 ^ rk[43];
}

// Keystream block (domain, index) as four little-endian words: the sixteen
// output bytes in order, i.e. eight little-endian 16-bit words.
LWE_DEV uint4 aes_ctr_block(const AesTab &tab, const uint32_t rk[44],
                            uint64_t domain, uint64_t index) {
  uint32_t s0 = bswap32((uint32_t)(domain >> 32));
  uint32_t s1 = bswap32((uint32_t)domain);
  uint32_t s2 = bswap32((uint32_t)(index >> 32));
  uint32_t s3 = bswap32((uint32_t)index);
  aes_encrypt(tab, rk, s0, s1, s2, s3);
  return make_uint4(s0, s1, s2, s3);
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
