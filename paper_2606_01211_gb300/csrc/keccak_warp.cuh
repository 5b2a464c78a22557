// keccak_warp.cuh -- Keccak-f[1600] and SHA3-256 (FIPS 202) with one state
// per warp: thread t < 25 holds lane (x, y) = (t % 5, t / 5), i.e. lane
// x + 5y of the state, as a 64-bit register; threads 25..31 mirror threads
// 0..6, so every shuffle source is a valid lane and the mirrors stay exact
// copies.  Each step of a round (FIPS 202 Sec. 3.2) becomes a few warp
// shuffles: theta gathers the column parities, rho/pi pulls the moved lane
// and rotates it by its offset, chi reads the two row neighbours.
//
// A permutation then costs one round's shuffle latency per round instead of
// one thread's 24 x ~190 dependent ALU instructions, so a single long
// message (the public key's tree hash) finishes several times sooner;
// batched hashing of many messages stays with one state per thread, which
// spends no instructions on data movement.
#pragma once
#include "keccak.cuh"

struct KeccakWarpMap {
  uint32_t col[4];  // the other four lanes of this lane's column (theta)
  uint32_t cm, cp;  // lanes (x - 1, y), (x + 1, y): C[x - 1], C[x + 1]
  uint32_t src;     // rho/pi: the lane (x', y') with (y', 2x' + 3y') = (x, y)
  uint32_t rot;     // rho offset of that lane
  uint32_t n1, n2;  // chi: lanes (x + 1, y), (x + 2, y)
  uint64_t rc_mask; // all-ones on lane (0, 0) (iota)
};

// rho offset of lane i = x + 5y: (t + 1)(t + 2) / 2 mod 64 where (x, y) is
// reached at step t of the walk (1, 0) -> (y, 2x + 3y); lane 0 has none.
LWE_DEV uint32_t keccak_rho_offset(uint32_t i) {
  uint32_t x = 1, y = 0;
  for (uint32_t t = 0; t < 24; t++) {
    if (x + 5 * y == i) return ((t + 1) * (t + 2) / 2) % 64;
    const uint32_t nx = y, ny = (2 * x + 3 * y) % 5;
    x = nx;
    y = ny;
  }
  return 0;
}

LWE_DEV KeccakWarpMap keccak_warp_map(uint32_t lane) {
  const uint32_t t = lane % 25, x = t % 5, y = t / 5;
  KeccakWarpMap m;
#pragma unroll
  for (uint32_t k = 0; k < 4; k++) m.col[k] = x + 5 * ((y + 1 + k) % 5);
  m.cm = (x + 4) % 5 + 5 * y;
  m.cp = (x + 1) % 5 + 5 * y;
  const uint32_t xs = (x + 3 * y) % 5, ys = x;  // source of (x, y) under pi
  m.src = xs + 5 * ys;
  m.rot = keccak_rho_offset(m.src);
  m.n1 = (x + 1) % 5 + 5 * y;
  m.n2 = (x + 2) % 5 + 5 * y;
  m.rc_mask = (t == 0) ? ~0ull : 0ull;
  return m;
}

LWE_DEV uint64_t shfl64(uint64_t v, uint32_t src) {
  return __shfl_sync(0xffffffffu, v, (int)src);
}

// 64-bit rotation by a run-time amount r in [0, 63]: a half swap for r >= 32,
// then two funnel shifts by r mod 32.
LWE_DEV uint64_t rotl64_var(uint64_t v, uint32_t r) {
  uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  const bool sw = (r & 32) != 0;
  const uint32_t a = sw ? hi : lo, b = sw ? lo : hi;
  const uint32_t s = r & 31;
  hi = __funnelshift_l(a, b, s);
  lo = __funnelshift_l(b, a, s);
  return ((uint64_t)hi << 32) | lo;
}

LWE_DEV uint64_t keccak_f1600_warp(const KeccakWarpMap &m, uint64_t v) {
#pragma unroll 1
  for (int round = 0; round < 24; ++round) {
    // theta: C[x] = XOR of column x; D[x] = C[x - 1] ^ ROT(C[x + 1], 1)
    const uint64_t c = v ^ shfl64(v, m.col[0]) ^ shfl64(v, m.col[1]) ^ shfl64(v, m.col[2]) ^
                       shfl64(v, m.col[3]);
    const uint64_t cm = shfl64(c, m.cm), cp = shfl64(c, m.cp);
    v ^= cm ^ ROTL64(cp, 1);
    // rho and pi: B[x, y] = ROT(A[x', y'], r[x', y'])
    const uint64_t b = rotl64_var(shfl64(v, m.src), m.rot);
    // chi, iota
    const uint64_t b1 = shfl64(b, m.n1), b2 = shfl64(b, m.n2);
    v = b ^ (~b1 & b2) ^ (kKeccakRC[round] & m.rc_mask);
  }
  return v;
}

// The 8-byte message word that lane `t` absorbs from block `blk` of a
// `len`-byte message at global address msg (8-byte aligned), with the SHA-3
// domain bits and pad10*1 of the last block folded in.  Lanes 17..24 (the
// capacity) and the mirrors absorb nothing.
LWE_DEV uint64_t sha3_warp_word(const uint8_t *msg, uint32_t len, uint32_t blk, uint32_t t) {
  if (t >= SHA3_RATE / 8) return 0;
  const uint32_t base = blk * SHA3_RATE + 8 * t;
  uint64_t w = 0;
  if (base + 8 <= len) {
    w = __ldg(reinterpret_cast<const uint64_t *>(msg + base));
  } else if (base < len) {
    for (uint32_t b = 0; b < len - base; b++) w |= (uint64_t)__ldg(msg + base + b) << (8 * b);
  }
  if (base <= len && len < base + 8) w ^= (uint64_t)0x06 << (8 * (len - base));
  if (t == SHA3_RATE / 8 - 1 && blk == len / SHA3_RATE) w ^= 0x8000000000000000ull;
  return w;
}

// SHA3-256 of a message of at most 8 blocks (len < 8 x 136 = 1088 bytes, so
// one 1024-byte chunk of the tree hash) by one warp: every lane loads all of
// its words first, so the loads overlap instead of preceding each
// permutation.  Returns this thread's lane of the final state (lanes 0..3
// hold the digest).
LWE_DEV uint64_t sha3_256_warp_chunk(const KeccakWarpMap &m, const uint8_t *msg, uint32_t len,
                                     uint32_t lane) {
  const uint32_t t = lane % 25, nblk = len / SHA3_RATE + 1;
  uint64_t w[8];
#pragma unroll
  for (uint32_t k = 0; k < 8; k++) w[k] = (k < nblk) ? sha3_warp_word(msg, len, k, t) : 0;
  uint64_t v = 0;
  for (uint32_t k = 0; k < nblk; k++) {
    v = keccak_f1600_warp(m, v ^ w[0]);
#pragma unroll
    for (int j = 0; j < 7; j++) w[j] = w[j + 1];  // constant indices: w stays in registers
  }
  return v;
}

// SHA3-256 of `len` bytes (a multiple of 8) of shared or global memory at an
// 8-byte aligned address, by one warp.
LWE_DEV uint64_t sha3_256_warp_mem(const KeccakWarpMap &m, const uint64_t *msg, uint32_t len,
                                   uint32_t lane) {
  const uint32_t t = lane % 25;
  uint64_t v = 0;
  for (uint32_t blk = 0; blk <= len / SHA3_RATE; blk++) {
    const uint32_t base = blk * SHA3_RATE + 8 * t;
    uint64_t w = 0;
    if (t < SHA3_RATE / 8) {
      if (base + 8 <= len) w = msg[base / 8];
      if (base == len) w ^= 0x06;
      if (t == SHA3_RATE / 8 - 1 && blk == len / SHA3_RATE) w ^= 0x8000000000000000ull;
    }
    v = keccak_f1600_warp(m, v ^ w);
  }
  return v;
}
