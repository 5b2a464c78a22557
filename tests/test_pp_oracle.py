"""Pins of the paper-profile oracle (oracle/pp.py): the KEM of Alg. 1-5 with
the parameter sets of Tab. 1 (odd q, a 256-bit message encrypted bit by
bit, binomial secret, Gaussian e / r / e1, centred-uniform e2, threshold
decoding).  Each pin checks the oracle against something other than
itself: closed-form distributions over every input word, hand-built inputs
with known outcomes, a brute-force triple loop, the round-trip property and
hashlib's SHA3-256."""
import hashlib
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import pp

TINY = pp.PParams(n=16, q=3329, sigma=2.3, k=3, clip=10)


def test_binomial_pmf_exact_over_every_byte():
    """eta = 3: P(x) = C(6, 3 + x) / 64 (the two top bits of a byte unused)."""
    x = pp.binomial_from_bytes(np.arange(256, dtype=np.uint8), 3)
    for v in range(-3, 4):
        assert int((x == v).sum()) == 4 * math.comb(6, 3 + v)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_centred_uniform_over_every_word(k):
    x = pp.uniform_from_words(np.arange(65536, dtype=np.uint16), k)
    assert x.min() == -k and x.max() == k
    counts = np.bincount(x + k)
    lo = 65536 // (2 * k + 1)
    assert set(counts.tolist()) <= {lo, lo + 1}


@pytest.mark.parametrize("sigma,clip", [(2.3, 10), (1.7, 7), (1.2, 5), (1.0, 4)])
def test_gaussian_sampler_matches_table_probabilities(sigma, clip):
    """Over all 65536 words the sampler's counts are the rounded CDF of the
    normal distribution: #|e| <= k = 2 round_half_up(2^15 P(|e| <= k))
    (every t appears twice, once per sign bit), and the numpy sampler
    agrees with the C oracle's on every word."""
    T = O.cdf_table(sigma, clip)
    assert T is not None
    w = np.arange(65536, dtype=np.uint16)
    e = pp.gaussian_from_words(w, T, clip)
    assert np.abs(e).max() == clip
    mass = [0.5 * (math.erf((k + 0.5) / sigma / math.sqrt(2)) - math.erf((k - 0.5) / sigma / math.sqrt(2)))
            for k in range(clip + 1)]
    z = mass[0] + 2 * sum(mass[1:])
    acc = 0.0
    for k in range(clip):
        acc += (mass[k] if k == 0 else 2 * mass[k]) / z
        assert int((np.abs(e) <= k).sum()) == 2 * math.floor(acc * 32768 + 0.5)
    some = w[::97]
    assert [pp.gaussian_from_words(np.array([x]), T, clip)[0] for x in some] == \
        [O.sample(int(x), T, clip) for x in some]


@pytest.mark.parametrize("q", [3329, 12289, 65537])
def test_rejection_sampler_of_A(q):
    """The acceptance bound is the largest multiple of q below 2^32, so an
    accepted word is exactly uniform mod q; a rejected word falls through
    to the next try, and an entry rejected by every try is 0."""
    limit = q * ((1 << 32) // q)
    assert limit % q == 0 and (1 << 32) - limit < q
    w1 = np.array([0, limit - 1, limit, (1 << 32) - 1, 5], np.uint32)
    w2 = np.array([7, 7, 9, limit, 6], np.uint32)
    w3 = np.array([1, 1, 1, (1 << 32) - 1, 1], np.uint32)
    got = pp.a_from_words([w1, w2, w3], q)
    assert got.tolist() == [0, (limit - 1) % q, 9, 0, 5]


def test_expand_A_range_and_balance():
    p = pp.PParams(n=256, q=12289, sigma=2.3, k=3, clip=10)
    A = pp.expand_A(bytes(range(16)), p)
    assert A.shape == (256, 256) and A.min() >= 0 and A.max() < p.q
    counts = np.bincount(A.reshape(-1) * 16 // p.q, minlength=16)
    exp = A.size / 16
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 40  # 15 degrees of freedom: p < 1e-3 above ~37.7


def test_encrypt_matches_a_triple_loop():
    """u_k = A^T r_k + e1_k and v_k = t^T r_k + e2_k + m_k floor(q/2), each
    entry recomputed with explicit loops from the same drawn noise."""
    p = TINY
    pk, sk, A = pp.keygen(p, bytes(range(32)), want_A=True)
    _, t = pp._unpack_pk(p, pk)
    m = bytes(range(32, 64))
    seed = bytes(range(100, 116))
    Ut, v = pp.encrypt(p, pk, m, seed)
    Rt = pp.gaussian(seed, 3, pp.MBITS * p.n, p).reshape(pp.MBITS, p.n)
    E1t = pp.gaussian(seed, 4, pp.MBITS * p.n, p).reshape(pp.MBITS, p.n)
    e2 = pp.uniform_from_words(pp._words16(seed, 5, pp.MBITS), p.k)
    bits = pp.message_bits(m)
    for k in (0, 1, 77, 255):
        for j in range(p.n):
            s_ = sum(int(A[i][j]) * int(Rt[k][i]) for i in range(p.n)) + int(E1t[k][j])
            assert Ut[k][j] == s_ % p.q
        s_ = sum(int(t[i]) * int(Rt[k][i]) for i in range(p.n)) + int(e2[k]) + int(bits[k]) * (p.q // 2)
        assert v[k] == s_ % p.q


def test_keygen_matches_a_triple_loop():
    p = TINY
    pk, sk, A = pp.keygen(p, bytes(range(32)), want_A=True)
    seedSE = hashlib.sha3_256(b"\x53" + bytes(range(32))).digest()[:16]
    s = pp.binomial_from_bytes(pp._bytes(seedSE, 1, p.n), 3)
    e = pp.gaussian(seedSE, 2, p.n, p)
    _, t = pp._unpack_pk(p, pk)
    for i in range(p.n):
        assert t[i] == (sum(int(A[i][j]) * int(s[j]) for j in range(p.n)) + int(e[i])) % p.q
    assert np.array_equal(np.frombuffer(sk[:p.n], np.int8), s.astype(np.int8))


def test_decode_thresholds_on_hand_built_ciphertexts():
    """With s = 0, mu = v: bit 1 exactly when q < 4 v < 3q."""
    p = TINY
    q = p.q
    vals = [0, q // 4, q // 4 + 1, q // 2, (3 * q) // 4, (3 * q) // 4 + 1, q - 1]
    v = np.array(vals + [0] * (pp.MBITS - len(vals)), np.int64)
    ct = pp.ct_bytes_of(np.zeros((pp.MBITS, p.n), np.int64), v)
    m = pp.decrypt(p, np.zeros(p.n, np.int64), ct)
    bits = pp.message_bits(m)[:len(vals)].tolist()
    assert bits == [int(q < 4 * x < 3 * q) for x in vals]
    assert bits == [0, 0, 1, 1, 1, 0, 0]


@pytest.mark.parametrize("name", ["PP512", "PP1024"])
def test_decrypt_inverts_encrypt(name):
    p = pp.preset(name)
    pk, sk, A = pp.keygen(p, bytes([7]) * 32, want_A=True)
    s = np.frombuffer(sk[:p.n], np.int8).astype(np.int64)
    r = np.random.default_rng(3)
    for i in range(3):
        m = r.integers(0, 256, 32, dtype=np.uint8).tobytes()
        Ut, v = pp.encrypt(p, pk, m, bytes([i]) * 16, A)
        assert pp.decrypt(p, s, pp.ct_bytes_of(Ut, v)) == m


def test_kem_round_trip_and_implicit_rejection():
    p = pp.preset("PP512")
    pk, sk, A = pp.keygen(p, bytes([9]) * 32, want_A=True)
    ct, K = pp.encaps(p, pk, bytes([1]) * 32, A)
    assert len(ct) == p.ct_bytes and len(pk) == p.pk_bytes and len(sk) == p.sk_bytes
    assert pp.decaps(p, sk, ct, A) == K
    m = hashlib.sha3_256(b"\x4d" + bytes([1]) * 32).digest()
    kp = hashlib.sha3_256(O.htree(pk) + m).digest()
    row = 4 * p.n
    hc = O.htree(b"".join([O.htree(ct[k * row:(k + 1) * row]) for k in range(256)] +
                          [O.htree(ct[256 * row:])]))
    assert hc == pp.hash_ct(p, ct)
    assert K == hashlib.sha3_256(kp + hc).digest()
    bad = bytearray(ct)
    bad[12345] ^= 4
    bad = bytes(bad)
    z = sk[p.n:p.n + 32]
    assert pp.decaps(p, sk, bad, A) == hashlib.sha3_256(z + pp.hash_ct(p, bad)).digest()


@pytest.mark.parametrize("q", [3329, 12289, 65537])
def test_expand_A_stream_layout_vs_library_ctr(q):
    """The counter-stream layout of A: entry (i, j) is little-endian 32-bit
    word i n + j of the AES-128-CTR stream of domain 16 (initial counter
    BE64(16) || BE64(0)), reduced mod q when below the acceptance bound;
    the keystream comes from an independent AES library here."""
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    n = 48
    p = pp.PParams(n=n, q=q, sigma=2.3, k=3, clip=10)
    seed = bytes(range(100, 116))
    iv = pp.A_DOMAIN.to_bytes(8, "big") + bytes(8)
    ks = ciphers.Cipher(ciphers.algorithms.AES(seed), ciphers.modes.CTR(iv)).encryptor().update(
        bytes(4 * n * n))
    w = np.frombuffer(ks, dtype="<u4").astype(np.int64)
    limit = q * ((1 << 32) // q)
    assert (w < limit).all()  # no entry of this seed falls through to domain 17
    assert np.array_equal(pp.expand_A(seed, p), (w % q).reshape(n, n))


def test_noise_stream_layout_vs_library_ctr():
    """The samplers' inputs: byte k (binomial s, domain 1) and little-endian
    16-bit word k (Gaussian e, r, e1 and uniform e2, domains 2-5) of the
    AES-128-CTR stream of their domain, taken from an independent AES
    library here."""
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    key = bytes(range(7, 23))
    for d in (1, 2, 3, 4, 5):
        iv = d.to_bytes(8, "big") + bytes(8)
        ks = ciphers.Cipher(ciphers.algorithms.AES(key), ciphers.modes.CTR(iv)).encryptor().update(
            bytes(1000))
        assert np.array_equal(pp._bytes(key, d, 999), np.frombuffer(ks, np.uint8)[:999])
        assert np.array_equal(pp._words16(key, d, 499), np.frombuffer(ks, "<u2")[:499])
        T = O.cdf_table(2.3, 10)
        assert np.array_equal(pp.gaussian(key, d, 499, TINY),
                              pp.gaussian_from_words(np.frombuffer(ks, "<u2")[:499], T, 10))
