"""The windowed AES-CTR rounds of the generators (aes_ctr_run and
aes_ctr_run_block in csrc/aes.cuh) restated in Python from FIPS-197: inside
a 256-aligned window of counter indices only the last input byte varies,
so the XOR of round 1's other 15 table lookups and of 12 of round 2's,
with their round keys, is the same for the whole window.  This checks that
the partial sums, recombined, are AES-128 itself: against the oracle's
AES-CTR block (oracle/lwe_oracle.c) for random keys, streams and windows,
including the window's first and last index and the last window of the
64-bit counter space.  The CUDA sequence itself is checked against the
oracle on the GPU (tests/test_gpu_probe.py, LWE_PROBE_AES_RUN)."""
import random

from oracle import oracle as O


def _gmul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a = ((a << 1) ^ (0x11B if a & 0x80 else 0)) & 0xFF
        b >>= 1
    return r


def _sbox():
    inv = [0] * 256
    for a in range(1, 256):
        inv[a] = next(b for b in range(1, 256) if _gmul(a, b) == 1)
    rot = lambda x, s: ((x << s) | (x >> (8 - s))) & 0xFF
    return [inv[x] ^ rot(inv[x], 1) ^ rot(inv[x], 2) ^ rot(inv[x], 3) ^ rot(inv[x], 4) ^ 0x63
            for x in range(256)]


S = _sbox()
# round table T0[x] = 2.S(x) | S(x) << 8 | S(x) << 16 | 3.S(x) << 24 and
# its byte rotations T1..T3 (little-endian columns)
T0 = [_gmul(S[x], 2) | S[x] << 8 | S[x] << 16 | _gmul(S[x], 3) << 24 for x in range(256)]
TK = [[((v << (8 * k)) | (v >> (32 - 8 * k))) & 0xFFFFFFFF if k else v for v in T0]
      for k in range(4)]


def T(k, byte, s):
    return TK[k][(s >> (8 * byte)) & 0xFF]


def bswap(v):
    return int.from_bytes(v.to_bytes(4, "little"), "big")


def key_expand(key):
    rk = [int.from_bytes(key[4 * i:4 * i + 4], "little") for i in range(4)]
    rcon = 1
    for i in range(4, 44):
        t = rk[i - 1]
        if i % 4 == 0:
            t = (S[(t >> 8) & 0xFF] | S[(t >> 16) & 0xFF] << 8 | S[t >> 24] << 16
                 | S[t & 0xFF] << 24) ^ rcon
            rcon = _gmul(rcon, 2)
        rk.append(rk[i - 4] ^ t)
    return rk


def rounds_from(rk, s, r0):
    """Rounds r0..9 of the table form, then the final round, on columns s."""
    s0, s1, s2, s3 = s
    for r in range(r0, 10):
        s0, s1, s2, s3 = (
            T(0, 0, s0) ^ T(1, 1, s1) ^ T(2, 2, s2) ^ T(3, 3, s3) ^ rk[4 * r],
            T(0, 0, s1) ^ T(1, 1, s2) ^ T(2, 2, s3) ^ T(3, 3, s0) ^ rk[4 * r + 1],
            T(0, 0, s2) ^ T(1, 1, s3) ^ T(2, 2, s0) ^ T(3, 3, s1) ^ rk[4 * r + 2],
            T(0, 0, s3) ^ T(1, 1, s0) ^ T(2, 2, s1) ^ T(3, 3, s2) ^ rk[4 * r + 3])
    cols = (s0, s1, s2, s3)
    out = b""
    for c in range(4):
        w = (S[cols[c] & 0xFF] | S[(cols[(c + 1) % 4] >> 8) & 0xFF] << 8
             | S[(cols[(c + 2) % 4] >> 16) & 0xFF] << 16 | S[cols[(c + 3) % 4] >> 24] << 24)
        out += (w ^ rk[40 + c]).to_bytes(4, "little")
    return out


def window(rk, domain, index):
    """The per-window partial sums (aes_ctr_run)."""
    s0 = bswap(domain >> 32) ^ rk[0]
    s1 = bswap(domain & 0xFFFFFFFF) ^ rk[1]
    s2 = bswap(index >> 32) ^ rk[2]
    s3 = bswap(index & 0xFFFFFF00) ^ rk[3]
    k0 = T(0, 0, s0) ^ T(1, 1, s1) ^ T(2, 2, s2) ^ rk[4]
    t1 = T(0, 0, s1) ^ T(1, 1, s2) ^ T(2, 2, s3) ^ T(3, 3, s0) ^ rk[5]
    t2 = T(0, 0, s2) ^ T(1, 1, s3) ^ T(2, 2, s0) ^ T(3, 3, s1) ^ rk[6]
    t3 = T(0, 0, s3) ^ T(1, 1, s0) ^ T(2, 2, s1) ^ T(3, 3, s2) ^ rk[7]
    return (s3, k0,
            T(1, 1, t1) ^ T(2, 2, t2) ^ T(3, 3, t3) ^ rk[8],
            T(0, 0, t1) ^ T(1, 1, t2) ^ T(2, 2, t3) ^ rk[9],
            T(0, 0, t2) ^ T(1, 1, t3) ^ T(3, 3, t1) ^ rk[10],
            T(0, 0, t3) ^ T(2, 2, t1) ^ T(3, 3, t2) ^ rk[11])


def window_block(rk, w, x):
    """Block (window base | x): one lookup of round 1, four of round 2."""
    s3, k0, k1, k2, k3, k4 = w
    t0 = k0 ^ T(3, 3, s3 ^ (x << 24))
    return rounds_from(rk, (T(0, 0, t0) ^ k1, T(3, 3, t0) ^ k2, T(2, 2, t0) ^ k3,
                            T(1, 1, t0) ^ k4), 3)


def full_block(rk, domain, index):
    s = (bswap(domain >> 32), bswap(domain & 0xFFFFFFFF), bswap(index >> 32),
         bswap(index & 0xFFFFFFFF))
    return rounds_from(rk, tuple(s[i] ^ rk[i] for i in range(4)), 1)


def test_table_rounds_are_aes():
    """FIPS-197 Appendix B: the table form of the cipher on the standard's
    example block."""
    key = bytes.fromhex("2b7e151628aed2a6abf7158809cf4f3c")
    rk = key_expand(key)
    pt = bytes.fromhex("3243f6a8885a308d313198a2e0370734")
    s = [int.from_bytes(pt[4 * i:4 * i + 4], "little") ^ rk[i] for i in range(4)]
    assert rounds_from(rk, s, 1) == bytes.fromhex("3925841d02dc09fbdc118597196a0b32")


def test_window_blocks_equal_the_oracle():
    rng = random.Random(5)
    for trial in range(24):
        key = bytes(rng.randrange(256) for _ in range(16))
        domain = rng.choice([0, 1, 3, 16, rng.randrange(1 << 64)])
        base = rng.choice([0, 256, rng.randrange(1 << 40) & ~0xFF, (1 << 64) - 256])
        rk = key_expand(key)
        w = window(rk, domain, base + rng.randrange(256))  # any index of the window
        for x in rng.sample(range(1, 255), 4) + [0, 255]:
            ref = O.ctr_stream(key, domain, base + x, 1).tobytes()
            assert full_block(rk, domain, base + x) == ref
            assert window_block(rk, w, x) == ref, (trial, x)
