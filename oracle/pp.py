"""Paper-profile oracle: the KEM of Alg. 1-5 with the parameter sets of
Tab. 1 -- odd q, one Regev encryption per message bit (a 256-bit message,
so Encrypt draws a 256-column r), a binomial secret, Gaussian e, r, e1 and a
centred-uniform e2, threshold decoding -- written plainly in numpy int64.

TEST INFRASTRUCTURE ONLY (like oracle.py): only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may use it.  It
shares no code with paper_2606_01211_gb300/; the AES-128 and SHA3-256
primitives are the C oracle's.

Readings, where the paper is silent or at odds with itself:

* Distributions follow Tab. 1: s binomial with eta = 3; e, r and e1
  Gaussian with the table's sigma; e2 centred uniform on [-k, k].  (Alg. 1
  and 2 write chi_eta for r and e1 as well; the table is the more specific
  statement.)
* Gaussian: the rounded-Gaussian CDF table of the matrix-form oracle
  (``oracle.cdf_table``) and its 16-bit sampler, clipped at |e| <= clip.
* Binomial eta = 3 from one keystream byte b:
  popcount(b & 7) - popcount((b >> 3) & 7).
* Centred uniform from a 16-bit word w: floor((2k + 1) w / 2^16) - k.
* A (Alg. 1, "sample(rho)"): uniform mod q by rejection.  Entry
  (i, j) takes 32-bit little-endian word i n + j of the stream (seedA,
  domain 16 + t); the word is accepted when w < q floor(2^32 / q), giving
  A = w mod q, else t + 1 is tried (t < 8).
* Streams (key, domain): s (seedSE, 1), e (seedSE, 2); Encrypt's r
  (seedSE', 3, row k of r^T = word k n + i), e1 (seedSE', 4, same layout),
  e2 (seedSE', 5, word k).  Sample k of a 16-bit stream is word k of the
  keystream, of a byte stream byte k.
* Seeds as in the matrix form: seedA, seedSE, z from SHA3-256 of a prefix
  byte and the master seed; m = SHA3-256(0x4D || coins), bit k = bit k % 8
  of byte k / 8; K' = H(pkh || m); seedSE' = H(0x01 || pkh || m)[0:16]
  derandomises Encrypt so that Decaps can re-encrypt (Alg. 5).
* Decode (Alg. 3): bit k is 1 iff q < 4 mu_k < 3q, i.e. 0 iff mu_k <= q/4
  or mu_k >= 3q/4.
* Layouts: pk = seedA || t (n uint32 LE); sk = s (n int8) || z || pkh ||
  pk; ct = U^T (256 x n uint32 LE, row k = u_k) || v (256 uint32 LE).  H is
  SHA3-256; H(pk) is the tree hash of the matrix form (``oracle.htree``),
  and H(c) = htree(htree(u_0) || ... || htree(u_255) || htree(v)), so that
  the multi-megabyte ciphertext needs no long sequential root.

Parity unpinned: the stream domains, seed prefixes and byte layouts above
are this project's readings, fixed only by this oracle.  (Given those
readings, the word layout of the A, r, e1 and e2 streams is pinned against
a library AES-CTR, tests/test_pp_oracle.py.)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import oracle as O

MBITS = 256
A_DOMAIN = 16
A_TRIES = 8


@dataclass(frozen=True)
class PParams:
    n: int
    q: int
    sigma: float
    k: int          # e2 bound
    clip: int       # Gaussian clip
    eta: int = 3

    @property
    def pk_bytes(self) -> int:
        return 16 + 4 * self.n

    @property
    def sk_bytes(self) -> int:
        return self.n + 64 + self.pk_bytes

    @property
    def ct_bytes(self) -> int:
        return 4 * MBITS * self.n + 4 * MBITS


def max_clip(sigma: float) -> int:
    """The largest clip (<= 15) for which the CDF table is valid."""
    c = 15
    while c > 1 and O.cdf_table(sigma, c) is None:
        c -= 1
    return c


def _pp(n, q, sigma, k):
    return PParams(n, q, sigma, k, max_clip(sigma))


# Tab. 1 (n, q, Gaussian sigma, centred-uniform k); eta = 3 throughout
PRESETS = {
    "PP512": (512, 3329, 2.3, 3),
    "PP1024": (1024, 12289, 2.3, 3),
    "PP2048": (2048, 12289, 2.3, 3),
    "PP4096": (4096, 12289, 1.7, 3),
    "PP8192": (8192, 65537, 1.2, 2),
    "PP16384": (16384, 65537, 1.2, 2),
    "PP32768": (32768, 65537, 1.0, 2),
}


def preset(name: str) -> PParams:
    return _pp(*PRESETS[name])


# ---- samplers ------------------------------------------------------------

def binomial_from_bytes(b: np.ndarray, eta: int = 3) -> np.ndarray:
    """Centred binomial: the difference of two sums of eta bits."""
    b = b.astype(np.int64)
    lo = np.zeros_like(b)
    hi = np.zeros_like(b)
    for i in range(eta):
        lo += (b >> i) & 1
        hi += (b >> (eta + i)) & 1
    return lo - hi


def uniform_from_words(w: np.ndarray, k: int) -> np.ndarray:
    return (((2 * k + 1) * w.astype(np.int64)) >> 16) - k


def gaussian_from_words(w: np.ndarray, T: np.ndarray, clip: int) -> np.ndarray:
    """The CDF sampler: t = w >> 1, |e| = #{i < clip : t > T[i]}, sign w & 1."""
    w = w.astype(np.int64)
    t = w >> 1
    mag = np.zeros_like(w)
    for i in range(clip):
        mag += (t > int(T[i])).astype(np.int64)
    return np.where(w & 1, -mag, mag)


def a_from_words(words_by_try: list, q: int) -> np.ndarray:
    """Rejection: the first accepted try of each entry (0 if none is)."""
    limit = q * ((1 << 32) // q)
    out = np.zeros(words_by_try[0].shape, np.int64)
    done = np.zeros(out.shape, bool)
    for w in words_by_try:
        w = w.astype(np.int64)
        take = (~done) & (w < limit)
        out[take] = w[take] % q
        done |= take
    return out


def _words16(key: bytes, domain: int, count: int) -> np.ndarray:
    return O.ctr_stream(key, domain, 0, (count + 7) // 8).view("<u2")[:count]


def _words32(key: bytes, domain: int, count: int) -> np.ndarray:
    return O.ctr_stream(key, domain, 0, (count + 3) // 4).view("<u4")[:count]


def _bytes(key: bytes, domain: int, count: int) -> np.ndarray:
    return O.ctr_stream(key, domain, 0, (count + 15) // 16)[:count]


def expand_A(seedA: bytes, p: PParams) -> np.ndarray:
    """A in Z_q^{n x n}, row-major (Alg. 1)."""
    n = p.n
    limit = p.q * ((1 << 32) // p.q)
    tries = [_words32(seedA, A_DOMAIN, n * n)]
    # a further try is drawn only while some entry has been rejected by all
    # earlier ones
    rejected = tries[0] >= limit
    while rejected.any() and len(tries) < A_TRIES:
        tries.append(_words32(seedA, A_DOMAIN + len(tries), n * n))
        rejected &= tries[-1] >= limit
    return a_from_words(tries, p.q).reshape(n, n)


def gaussian(key: bytes, domain: int, count: int, p: PParams) -> np.ndarray:
    T = O.cdf_table(p.sigma, p.clip)
    return gaussian_from_words(_words16(key, domain, count), T, p.clip)


# ---- the scheme ------------------------------------------------------------

def _h(b: bytes) -> bytes:
    return O.sha3_256(b)


def _u32le(a: np.ndarray) -> bytes:
    return np.ascontiguousarray(a, "<u4").tobytes()


def keygen(p: PParams, ms: bytes, want_A: bool = False):
    """Alg. 1: t = A s + e (mod q); pk = seedA || t, sk = s || z || pkh || pk."""
    seedA = _h(b"\x41" + ms)[:16]
    seedSE = _h(b"\x53" + ms)[:16]
    z = _h(b"\x5a" + ms)
    A = expand_A(seedA, p)
    s = binomial_from_bytes(_bytes(seedSE, 1, p.n), p.eta)
    e = gaussian(seedSE, 2, p.n, p)
    t = (A.astype(np.float64) @ s.astype(np.float64)).astype(np.int64)  # exact: |sum| < 2^53
    t = (t + e) % p.q
    pk = seedA + _u32le(t)
    sk = s.astype(np.int8).tobytes() + z + O.htree(pk) + pk
    return (pk, sk, A) if want_A else (pk, sk)


def _unpack_pk(p: PParams, pk: bytes):
    return pk[:16], np.frombuffer(pk[16:16 + 4 * p.n], "<u4").astype(np.int64)


def message_bits(m: bytes) -> np.ndarray:
    b = np.frombuffer(m, np.uint8)
    return np.array([(b[k // 8] >> (k % 8)) & 1 for k in range(MBITS)], np.int64)


def encrypt(p: PParams, pk: bytes, m: bytes, seed: bytes, A: np.ndarray | None = None):
    """Alg. 2 for each of the 256 message bits: with r_k, e1_k, e2_k drawn
    from seed, u_k = A^T r_k + e1_k and v_k = t^T r_k + e2_k + m_k floor(q/2)
    (mod q).  Returns (U^T as 256 x n, v)."""
    n, q = p.n, p.q
    seedA, t = _unpack_pk(p, pk)
    if A is None:
        A = expand_A(seedA, p)
    Rt = gaussian(seed, 3, MBITS * n, p).reshape(MBITS, n)     # row k = r_k
    E1t = gaussian(seed, 4, MBITS * n, p).reshape(MBITS, n)    # row k = e1_k
    e2 = uniform_from_words(_words16(seed, 5, MBITS), p.k)
    Ut = (Rt.astype(np.float64) @ A.astype(np.float64)).astype(np.int64)  # r_k^T A = (A^T r_k)^T
    Ut = (Ut + E1t) % q
    v = (Rt.astype(np.float64) @ t.astype(np.float64)).astype(np.int64)
    v = (v + e2 + message_bits(m) * (q // 2)) % q
    return Ut, v


def ct_bytes_of(Ut: np.ndarray, v: np.ndarray) -> bytes:
    return _u32le(Ut.reshape(-1)) + _u32le(v)


def decrypt(p: PParams, s: np.ndarray, ct: bytes) -> bytes:
    """Alg. 3: mu_k = v_k - s^T u_k (mod q); bit 1 iff q < 4 mu_k < 3q."""
    n, q = p.n, p.q
    Ut = np.frombuffer(ct[:4 * MBITS * n], "<u4").astype(np.int64).reshape(MBITS, n)
    v = np.frombuffer(ct[4 * MBITS * n:], "<u4").astype(np.int64)
    mu = (v - (Ut.astype(np.float64) @ s.astype(np.float64)).astype(np.int64)) % q
    bits = ((4 * mu > q) & (4 * mu < 3 * q)).astype(np.uint8)
    out = bytearray(32)
    for k in range(MBITS):
        out[k // 8] |= int(bits[k]) << (k % 8)
    return bytes(out)


def hash_ct(p: PParams, ct: bytes) -> bytes:
    """H(c): the tree hash of the rows' and v's tree hashes."""
    row = 4 * p.n
    parts = [O.htree(ct[k * row:(k + 1) * row]) for k in range(MBITS)]
    parts.append(O.htree(ct[MBITS * row:]))
    return O.htree(b"".join(parts))


def _derive(pkh: bytes, m: bytes):
    return _h(pkh + m), _h(b"\x01" + pkh + m)[:16]


def encaps(p: PParams, pk: bytes, coins: bytes, A: np.ndarray | None = None):
    """Alg. 4: m from the coins, c = Encrypt(pk, m), K = H(K' || H(c))."""
    m = _h(b"\x4d" + coins)
    pkh = O.htree(pk)
    kp, seed = _derive(pkh, m)
    Ut, v = encrypt(p, pk, m, seed, A)
    ct = ct_bytes_of(Ut, v)
    return ct, _h(kp + hash_ct(p, ct))


def decaps(p: PParams, sk: bytes, ct: bytes, A: np.ndarray | None = None) -> bytes:
    """Alg. 5: m' = Decrypt(sk, c), c' = Encrypt(pk, m'), K = H(K' || H(c))
    if c' = c, else H(z || H(c))."""
    n = p.n
    s = np.frombuffer(sk[:n], np.int8).astype(np.int64)
    z, pkh, pk = sk[n:n + 32], sk[n + 32:n + 64], sk[n + 64:]
    m = decrypt(p, s, ct)
    kp, seed = _derive(pkh, m)
    Ut, v = encrypt(p, pk, m, seed, A)
    hc = hash_ct(p, ct)
    return _h((kp if ct_bytes_of(Ut, v) == ct else z) + hc)
