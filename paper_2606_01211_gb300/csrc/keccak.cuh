// keccak.cuh -- Keccak-f[1600] and SHA3-256 (FIPS 202), one state per thread.
//
// H of the paper's Alg. 4-5 is left unnamed; this library uses SHA3-256.
// Each thread holds a full 25-lane state in registers and absorbs its own
// message, so independent messages (one per encapsulation, or one per
// 1024-byte chunk of a long message) run in parallel across threads.
#pragma once
#include "common.cuh"

__constant__ uint64_t kKeccakRC[24] = {
    0x0000000000000001ull, 0x0000000000008082ull, 0x800000000000808Aull,
    0x8000000080008000ull, 0x000000000000808Bull, 0x0000000080000001ull,
    0x8000000080008081ull, 0x8000000000008009ull, 0x000000000000008Aull,
    0x0000000000000088ull, 0x0000000080008009ull, 0x000000008000000Aull,
    0x000000008000808Bull, 0x800000000000008Bull, 0x8000000000008089ull,
    0x8000000000008003ull, 0x8000000000008002ull, 0x8000000000000080ull,
    0x000000000000800Aull, 0x800000008000000Aull, 0x8000000080008081ull,
    0x8000000000008080ull, 0x0000000080000001ull, 0x8000000080008008ull};

// 64-bit rotation; compiles to a pair of funnel shifts.  (Rotations written
// as multiply-adds to unload the integer ALU pipe were measured slower: more
// instructions and longer dependency chains.)
#define ROTL64(x, r) (((x) << (r)) | ((x) >> (64 - (r))))

// Keccak-f[1600]: 24 rounds of theta, rho, pi, chi, iota.  Lane (x, y) is
// s[x + 5y]; rho/pi move lane (x, y), rotated by its offset, to (y, 2x+3y).
LWE_DEV void keccak_f1600(uint64_t s[25]) {
#pragma unroll 1
  for (int round = 0; round < 24; ++round) {
    uint64_t C0 = s[0] ^ s[5] ^ s[10] ^ s[15] ^ s[20];
    uint64_t C1 = s[1] ^ s[6] ^ s[11] ^ s[16] ^ s[21];
    uint64_t C2 = s[2] ^ s[7] ^ s[12] ^ s[17] ^ s[22];
    uint64_t C3 = s[3] ^ s[8] ^ s[13] ^ s[18] ^ s[23];
    uint64_t C4 = s[4] ^ s[9] ^ s[14] ^ s[19] ^ s[24];
    uint64_t D0 = C4 ^ ROTL64(C1, 1);
    uint64_t D1 = C0 ^ ROTL64(C2, 1);
    uint64_t D2 = C1 ^ ROTL64(C3, 1);
    uint64_t D3 = C2 ^ ROTL64(C4, 1);
    uint64_t D4 = C3 ^ ROTL64(C0, 1);
    uint64_t b[25];
    b[0] = s[0] ^ D0;
    b[10] = ROTL64(s[1] ^ D1, 1);
    b[20] = ROTL64(s[2] ^ D2, 62);
    b[5] = ROTL64(s[3] ^ D3, 28);
    b[15] = ROTL64(s[4] ^ D4, 27);
    b[16] = ROTL64(s[5] ^ D0, 36);
    b[1] = ROTL64(s[6] ^ D1, 44);
    b[11] = ROTL64(s[7] ^ D2, 6);
    b[21] = ROTL64(s[8] ^ D3, 55);
    b[6] = ROTL64(s[9] ^ D4, 20);
    b[7] = ROTL64(s[10] ^ D0, 3);
    b[17] = ROTL64(s[11] ^ D1, 10);
    b[2] = ROTL64(s[12] ^ D2, 43);
    b[12] = ROTL64(s[13] ^ D3, 25);
    b[22] = ROTL64(s[14] ^ D4, 39);
    b[23] = ROTL64(s[15] ^ D0, 41);
    b[8] = ROTL64(s[16] ^ D1, 45);
    b[18] = ROTL64(s[17] ^ D2, 15);
    b[3] = ROTL64(s[18] ^ D3, 21);
    b[13] = ROTL64(s[19] ^ D4, 8);
    b[14] = ROTL64(s[20] ^ D0, 18);
    b[24] = ROTL64(s[21] ^ D1, 2);
    b[9] = ROTL64(s[22] ^ D2, 61);
    b[19] = ROTL64(s[23] ^ D3, 56);
    b[4] = ROTL64(s[24] ^ D4, 14);
#pragma unroll
    for (int y = 0; y < 25; y += 5) {
      s[y + 0] = b[y + 0] ^ (~b[y + 1] & b[y + 2]);
      s[y + 1] = b[y + 1] ^ (~b[y + 2] & b[y + 3]);
      s[y + 2] = b[y + 2] ^ (~b[y + 3] & b[y + 4]);
      s[y + 3] = b[y + 3] ^ (~b[y + 4] & b[y + 0]);
      s[y + 4] = b[y + 4] ^ (~b[y + 0] & b[y + 1]);
    }
    s[0] ^= kKeccakRC[round];
  }
}

#define SHA3_RATE 136

LWE_DEV void sha3_init(uint64_t s[25]) {
#pragma unroll
  for (int i = 0; i < 25; i++) s[i] = 0;
}

LWE_DEV void sha3_digest(const uint64_t s[25], uint8_t *out) {
  // out may be any alignment
#pragma unroll
  for (int i = 0; i < 4; i++) {
    uint64_t v = s[i];
#pragma unroll
    for (int b = 0; b < 8; b++) out[8 * i + b] = (uint8_t)(v >> (8 * b));
  }
}

LWE_DEV void sha3_digest16(const uint64_t s[25], uint8_t *out16) {
  // first 16 bytes, destination 16-byte aligned
  *reinterpret_cast<uint4 *>(out16) =
      make_uint4((uint32_t)s[0], (uint32_t)(s[0] >> 32), (uint32_t)s[1],
                 (uint32_t)(s[1] >> 32));
}

// SHA3-256 of `len` bytes at global address msg, which must be 8-byte
// aligned: whole lanes are loaded with 64-bit reads and every state index is
// a compile-time constant (the state stays in registers).
LWE_DEV void sha3_256_global(const uint8_t *msg, uint32_t len, uint64_t s[25]) {
  sha3_init(s);
  const uint64_t *p = reinterpret_cast<const uint64_t *>(msg);
  uint32_t off = 0;
  while (len - off >= SHA3_RATE) {
#pragma unroll
    for (int i = 0; i < SHA3_RATE / 8; i++) s[i] ^= __ldg(p + off / 8 + i);
    keccak_f1600(s);
    off += SHA3_RATE;
  }
  // final partial block with pad10*1 and the SHA-3 domain bits
  const uint32_t rem = len - off;
#pragma unroll
  for (int i = 0; i < SHA3_RATE / 8; i++) {
    const uint32_t base = 8 * i;
    uint64_t lane = 0;
    if (base + 8 <= rem) {
      lane = __ldg(p + off / 8 + i);
    } else if (base < rem) {
      for (uint32_t b = 0; b < rem - base; b++) lane |= (uint64_t)msg[off + base + b] << (8 * b);
    }
    if (base <= rem && rem < base + 8) lane ^= (uint64_t)0x06 << (8 * (rem - base));
    if (i == SHA3_RATE / 8 - 1) lane ^= 0x8000000000000000ull;
    s[i] ^= lane;
  }
  keccak_f1600(s);
}

// Absorb (and permute) blocks j0 .. j1-1 of the padded SHA3-256 input of a
// `len`-byte message at global address msg (8-byte aligned): block j holds
// bytes [136 j, 136 j + 136); block len / 136, the last, holds the rest with
// the padding.  sha3_256_global is sha3_init and then blocks 0 .. len / 136;
// a sponge can so be advanced in pieces, by different threads in turn.
LWE_DEV void sha3_absorb_global(const uint8_t *msg, uint32_t len, uint32_t j0, uint32_t j1,
                                uint64_t s[25]) {
  const uint64_t *p = reinterpret_cast<const uint64_t *>(msg);
  const uint32_t full = len / SHA3_RATE;
  for (uint32_t j = j0; j < j1; j++) {
    const uint32_t off = j * SHA3_RATE;
    if (j < full) {
#pragma unroll
      for (int i = 0; i < SHA3_RATE / 8; i++) s[i] ^= __ldg(p + off / 8 + i);
    } else {
      const uint32_t rem = len - off;
#pragma unroll
      for (int i = 0; i < SHA3_RATE / 8; i++) {
        const uint32_t base = 8 * i;
        uint64_t lane = 0;
        if (base + 8 <= rem) {
          lane = __ldg(p + off / 8 + i);
        } else if (base < rem) {
          for (uint32_t b = 0; b < rem - base; b++)
            lane |= (uint64_t)msg[off + base + b] << (8 * b);
        }
        if (base <= rem && rem < base + 8) lane ^= (uint64_t)0x06 << (8 * (rem - base));
        if (i == SHA3_RATE / 8 - 1) lane ^= 0x8000000000000000ull;
        s[i] ^= lane;
      }
    }
    keccak_f1600(s);
  }
}

// The same for a message in shared or global memory read with generic
// loads (len a multiple of 8).
LWE_DEV void sha3_absorb_mem(const uint8_t *msg, uint32_t len, uint32_t j0, uint32_t j1,
                             uint64_t s[25]) {
  const uint64_t *p = reinterpret_cast<const uint64_t *>(msg);
  const uint32_t full = len / SHA3_RATE;
  for (uint32_t j = j0; j < j1; j++) {
    const uint32_t off = j * SHA3_RATE;
    if (j < full) {
#pragma unroll
      for (int i = 0; i < SHA3_RATE / 8; i++) s[i] ^= p[off / 8 + i];
    } else {
      const uint32_t rem = len - off;
#pragma unroll
      for (int i = 0; i < SHA3_RATE / 8; i++) {
        const uint32_t base = 8 * i;
        uint64_t lane = (base + 8 <= rem) ? p[off / 8 + i] : 0;
        if (base == rem) lane ^= 0x06;
        if (i == SHA3_RATE / 8 - 1) lane ^= 0x8000000000000000ull;
        s[i] ^= lane;
      }
    }
    keccak_f1600(s);
  }
}

// SHA3-256 of `len` bytes at an 8-byte aligned address in shared or global
// memory (generic loads; len a multiple of 8).
LWE_DEV void sha3_256_mem(const uint8_t *msg, uint32_t len, uint64_t s[25]) {
  sha3_init(s);
  const uint64_t *p = reinterpret_cast<const uint64_t *>(msg);
  uint32_t off = 0;
  while (len - off >= SHA3_RATE) {
#pragma unroll
    for (int i = 0; i < SHA3_RATE / 8; i++) s[i] ^= p[off / 8 + i];
    keccak_f1600(s);
    off += SHA3_RATE;
  }
  const uint32_t rem = len - off;
#pragma unroll
  for (int i = 0; i < SHA3_RATE / 8; i++) {
    const uint32_t base = 8 * i;
    uint64_t lane = (base + 8 <= rem) ? p[off / 8 + i] : 0;
    if (base == rem) lane ^= 0x06;
    if (i == SHA3_RATE / 8 - 1) lane ^= 0x8000000000000000ull;
    s[i] ^= lane;
  }
  keccak_f1600(s);
}

// SHA3-256 of a short message (< 136 bytes) given as little-endian lanes
// already holding the message bytes (the rest zero); `len` in bytes.
LWE_DEV void sha3_256_lanes(uint64_t lanes[SHA3_RATE / 8], uint32_t len,
                            uint64_t s[25]) {
  lanes[len >> 3] ^= (uint64_t)0x06 << (8 * (len & 7));
  lanes[SHA3_RATE / 8 - 1] ^= 0x8000000000000000ull;
#pragma unroll
  for (int i = 0; i < 25; i++) s[i] = (i < SHA3_RATE / 8) ? lanes[i] : 0;
  keccak_f1600(s);
}

// Put `len` bytes at byte offset `pos` of a little-endian lane array.
LWE_DEV void lanes_put(uint64_t *lanes, uint32_t pos, const uint8_t *src,
                       uint32_t len) {
  for (uint32_t i = 0; i < len; i++)
    lanes[(pos + i) >> 3] |= (uint64_t)src[i] << (8 * ((pos + i) & 7));
}
LWE_DEV void lanes_put_u64(uint64_t *lanes, uint32_t pos, const uint64_t *src,
                           uint32_t nwords) {
  // pos must be a multiple of 8
  for (uint32_t i = 0; i < nwords; i++) lanes[(pos >> 3) + i] |= src[i];
}
LWE_DEV void lanes_zero(uint64_t *lanes) {
#pragma unroll
  for (int i = 0; i < SHA3_RATE / 8; i++) lanes[i] = 0;
}
