"""Pins of the CPU oracle to things other than itself.

Each test checks the oracle against a value the standards or the mathematics
fix: published worked examples (tests/golden/), independent library
implementations (hashlib, an independent AES, numpy integer matmul, the
normal CDF of scipy), closed forms, invariants of the KEM (Alg. 1-5 of the
paper) and brute force on tiny inputs.  None of them calls the CUDA path.
"""
import hashlib
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_01211_gb300.inputs import PRESETS, coins, master_seeds, random_bytes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _params(name, **over):
    d = dict(PRESETS[name])
    d.update(over)
    return O.Params(**d)


# ---------------------------------------------------------------- AES-128 --

def test_aes_fips197_worked_examples():
    rows = _golden("aes128_fips197.txt")
    assert len(rows) == 2
    for key, pt, ct in rows:
        assert O.aes128_encrypt(bytes.fromhex(key), bytes.fromhex(pt)).hex() == ct


def _aes_lib():
    mod = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    return mod


def test_aes_random_vs_independent_library():
    ciphers = _aes_lib()
    r = random_bytes(64, 32, 11)
    for row in r:
        key, blk = bytes(row[:16]), bytes(row[16:])
        enc = ciphers.Cipher(ciphers.algorithms.AES(key), ciphers.modes.ECB()).encryptor()
        assert O.aes128_encrypt(key, blk) == enc.update(blk)


def test_ctr_counter_format_vs_library_ctr_mode():
    """Block (d, b) is AES_k(BE64(d) || BE64(b)): a standard big-endian
    128-bit counter mode whose initial counter is BE64(d) || BE64(b0)."""
    ciphers = _aes_lib()
    key = bytes(random_bytes(1, 16, 12)[0])
    for d, b0 in [(0, 0), (3, 12345), (5, 2**40 + 7)]:
        iv = d.to_bytes(8, "big") + b0.to_bytes(8, "big")
        enc = ciphers.Cipher(ciphers.algorithms.AES(key), ciphers.modes.CTR(iv)).encryptor()
        ref = enc.update(bytes(16 * 9))
        assert O.ctr_blocks(key, d, b0, 9) == ref


# --------------------------------------------------------------- SHA3-256 --

def test_sha3_nist_examples():
    for msg, dig in _golden("sha3_256_fips202.txt"):
        m = b"" if msg == "-" else bytes.fromhex(msg)
        assert O.sha3_256(m).hex() == dig


@pytest.mark.parametrize("length", [0, 1, 31, 32, 64, 135, 136, 137, 271, 272, 273, 1000, 4097])
def test_sha3_vs_hashlib(length):
    m = bytes(random_bytes(1, max(length, 1), 100 + length)[0][:length])
    assert O.sha3_256(m) == hashlib.sha3_256(m).digest()


@pytest.mark.parametrize("length", [1, 1023, 1024, 1025, 5000, 10256, 15744])
def test_tree_hash_vs_hashlib_composition(length):
    m = bytes(random_bytes(1, length, 200 + length)[0])
    chunks = [m[i:i + O.TREE_CHUNK] for i in range(0, len(m), O.TREE_CHUNK)]
    ref = hashlib.sha3_256(b"".join(hashlib.sha3_256(c).digest() for c in chunks)).digest()
    assert O.htree(m) == ref


# ------------------------------------------------------------ CDF sampler --

def _gauss_mass(sigma, clip):
    stats = pytest.importorskip("scipy.stats")
    k = np.arange(0, clip + 1)
    p = stats.norm.cdf((k + 0.5) / sigma) - stats.norm.cdf((k - 0.5) / sigma)
    total = p[0] + 2 * p[1:].sum()
    return p / total


@pytest.mark.parametrize("name", ["P640", "P976", "P1344"])
def test_cdf_table_matches_gaussian_mass(name):
    cfg = PRESETS[name]
    T = O.cdf_table(cfg["sigma"], cfg["clip"]).astype(np.int64)
    assert np.all(np.diff(T) > 0)
    assert T[-1] < 32767
    # probability of |e| = k under the table: (T[k] - T[k-1]) / 2^15
    edges = np.concatenate([[-1], T, [32767]])
    prob_mag = np.diff(edges) / 32768.0
    p = _gauss_mass(cfg["sigma"], cfg["clip"])
    ref = np.concatenate([[p[0]], 2 * p[1:]])
    # each cumulative value is rounded to 1/2^15, so each cell is within 1/2^15
    assert np.max(np.abs(prob_mag - ref)) <= 1.0 / 32768 + 1e-12


@pytest.mark.parametrize("name", ["P640", "P976", "P1344"])
def test_sampler_exhaustive_over_all_words(name):
    cfg = PRESETS[name]
    c = cfg["clip"]
    T = O.cdf_table(cfg["sigma"], c)
    vals = np.array([O.sample(w, T, c) for w in range(65536)])
    assert vals.min() >= -c and vals.max() <= c
    hist = np.array([(vals == e).sum() for e in range(-c, c + 1)])
    assert np.array_equal(hist, hist[::-1])              # symmetric
    assert hist.sum() == 65536
    # frequencies follow the rounded Gaussian within the table's rounding
    p = _gauss_mass(cfg["sigma"], c)
    freq_mag = np.concatenate([[hist[c]], hist[c + 1:] + hist[:c][::-1]]) / 65536.0
    ref = np.concatenate([[p[0]], 2 * p[1:]])
    assert np.max(np.abs(freq_mag - ref)) <= 1.0 / 32768 + 1e-12
    # variance close to sigma^2 + 1/12 (rounding of a continuous Gaussian)
    var = (vals.astype(np.float64) ** 2).mean()
    assert abs(var - (cfg["sigma"] ** 2 + 1 / 12)) < 0.02 * cfg["sigma"] ** 2


def test_noise_stream_indexing_vs_library_ctr():
    """Sample k of stream (key, d) uses word k mod 8 of block k/8."""
    ciphers = _aes_lib()
    cfg = PRESETS["P976"]
    T = O.cdf_table(cfg["sigma"], cfg["clip"])
    key = bytes(random_bytes(1, 16, 13)[0])
    d = 4
    cnt = 8 * 37 + 5
    got = O.noise(key, d, T, cfg["clip"], cnt)
    iv = d.to_bytes(8, "big") + (0).to_bytes(8, "big")
    ks = ciphers.Cipher(ciphers.algorithms.AES(key), ciphers.modes.CTR(iv)).encryptor().update(
        bytes(16 * ((cnt + 7) // 8)))
    words = np.frombuffer(ks, dtype="<u2")[:cnt]
    T64 = T.astype(np.int64)
    t = (words >> 1).astype(np.int64)
    mag = (t[:, None] > T64[None, :]).sum(axis=1)
    ref = np.where(words & 1, -mag, mag)
    assert np.array_equal(got.astype(np.int64), ref)


# ---------------------------------------------------------------- matrices --

@pytest.mark.parametrize("n,logq", [(16, 16), (40, 15), (64, 16)])
def test_expand_A_vs_library_ctr(n, logq):
    ciphers = _aes_lib()
    seed = bytes(random_bytes(1, 16, 14 + n)[0])
    A = O.expand_A(seed, n, logq)
    iv = bytes(16)
    ks = ciphers.Cipher(ciphers.algorithms.AES(seed), ciphers.modes.CTR(iv)).encryptor().update(
        bytes(2 * n * n))
    ref = (np.frombuffer(ks, dtype="<u2") & ((1 << logq) - 1)).reshape(n, n)
    assert np.array_equal(A, ref)


@pytest.mark.parametrize("n,k,logq", [(8, 8, 16), (16, 8, 15), (32, 16, 16), (64, 24, 16)])
def test_products_brute_force(n, k, logq):
    r = np.random.default_rng(n * 100 + k)
    A = r.integers(0, 1 << logq, size=(n, n), dtype=np.uint16)
    St = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    E = r.integers(-12, 13, size=(n, k), dtype=np.int8)
    q = 1 << logq
    ref = (A.astype(np.int64) @ St.T.astype(np.int64) + E) % q
    assert np.array_equal(O.mul_AS(A, St, E, logq).astype(np.int64), ref)
    S = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    E2 = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    ref2 = (S.astype(np.int64) @ A.astype(np.int64) + E2) % q
    assert np.array_equal(O.mul_SA(S, A, E2, logq).astype(np.int64), ref2)
    assert np.array_equal(O.mul_SA(S, A, None, logq).astype(np.int64),
                          (S.astype(np.int64) @ A.astype(np.int64)) % q)


def test_products_special_cases():
    n, logq = 48, 16
    r = np.random.default_rng(5)
    A = r.integers(0, 1 << 16, size=(n, n), dtype=np.uint16)
    # a unit vector in S selects a column of A (A S) or a row of A (S A)
    St = np.zeros((8, n), np.int8)
    for c in range(8):
        St[c, 5 * c + 1] = 1
    out = O.mul_AS(A, St, None, logq)
    for c in range(8):
        assert np.array_equal(out[:, c], A[:, 5 * c + 1])
    out2 = O.mul_SA(St, A, None, logq)
    for c in range(8):
        assert np.array_equal(out2[c], A[5 * c + 1])
    # S = 0 leaves the error term (mod q)
    E = r.integers(-12, 13, size=(n, 8), dtype=np.int8)
    z = O.mul_AS(A, np.zeros((8, n), np.int8), E, logq)
    assert np.array_equal(z.astype(np.int64), E.astype(np.int64) % (1 << logq))
    # all-ones A gives the column sums of S, reduced mod q
    ones = np.ones((n, n), np.uint16)
    S = r.integers(-12, 13, size=(8, n), dtype=np.int8)
    cs = O.mul_SA(S, ones, None, logq)
    for c in range(8):
        assert np.all(cs[c].astype(np.int64) == int(S[c].astype(np.int64).sum()) % (1 << logq))


# --------------------------------------------------------------------- KEM --

def _unpack_pk(p, pk):
    B = np.frombuffer(pk[16:].tobytes(), dtype="<u2").reshape(p.n, 8)
    return bytes(pk[:16]), B


@pytest.mark.parametrize("name,count", [("P640", 12), ("P976", 6), ("P1344", 4)])
def test_kem_roundtrip_and_public_key_noise_bound(name, count):
    p = _params(name)
    ms = master_seeds(3, seed=7)
    cs = coins(count, seed=7)
    for i in range(3):
        pk, sk, A = O.keygen(p, bytes(ms[i]), want_A=True)
        seedA, B = _unpack_pk(p, pk)
        # A is the expansion of the seed stored in pk
        assert np.array_equal(A, O.expand_A(seedA, p.n, p.logq))
        # |B - A S| <= c elementwise (Eq. 1 with small e)
        St = sk[:8 * p.n].view(np.int8).reshape(8, p.n)
        q = 1 << p.logq
        e = (B.astype(np.int64) - A.astype(np.int64) @ St.T.astype(np.int64)) % q
        e = np.where(e >= q // 2, e - q, e)
        assert np.abs(e).max() <= p.clip
        # sk layout: S^T || z || H(pk) || pk
        assert bytes(sk[8 * p.n + 32:8 * p.n + 64]) == O.htree(bytes(pk))
        assert np.array_equal(sk[8 * p.n + 64:], pk)
        for j in range(count if i == 0 else 2):
            ct, K = O.encaps(p, pk, bytes(cs[j]))
            assert np.array_equal(O.decaps(p, sk, ct), K)
            assert np.array_equal(O.decaps(p, sk, ct, A=A), K)


def test_key_derivation_vs_hashlib():
    """K = H(H(pk || mu)-chain) of Alg. 4 re-derived with hashlib from the
    traced mu, pk and ct."""
    p = _params("P640")
    pk, sk = O.keygen(p, bytes(master_seeds(1, 3)[0]))
    c = bytes(coins(1, 3)[0])
    ct, K, tr = O.encaps(p, pk, c, trace=True)
    mub = O.sizes(p)[3]
    mu = hashlib.sha3_256(b"\x4d" + c).digest()[:mub]
    assert tr["mu"] == mu

    def tree(x):
        ch = [x[i:i + O.TREE_CHUNK] for i in range(0, len(x), O.TREE_CHUNK)]
        return hashlib.sha3_256(b"".join(hashlib.sha3_256(y).digest() for y in ch)).digest()

    pkh = tree(bytes(pk))
    kp = hashlib.sha3_256(pkh + mu).digest()
    assert tr["kprime"] == kp
    assert tr["seed_se"] == hashlib.sha3_256(b"\x01" + pkh + mu).digest()[:16]
    assert bytes(K) == hashlib.sha3_256(kp + tree(bytes(ct))).digest()
    # the keygen seeds follow the stated domain bytes
    ms = bytes(master_seeds(1, 3)[0])
    assert bytes(pk[:16]) == hashlib.sha3_256(b"\x41" + ms).digest()[:16]
    assert bytes(sk[8 * p.n:8 * p.n + 32]) == hashlib.sha3_256(b"\x5a" + ms).digest()


@pytest.mark.parametrize("where", ["Bprime", "C", "last"])
def test_implicit_rejection_key(where):
    """A ciphertext that does not re-encrypt to itself yields H(z || H(c))
    (Alg. 5, implicit rejection)."""
    p = _params("P640")
    pk, sk = O.keygen(p, bytes(master_seeds(1, 4)[0]))
    ct, K = O.encaps(p, pk, bytes(coins(1, 4)[0]))
    bad = ct.copy()
    pos = {"Bprime": 17, "C": 2 * 8 * p.n + 3, "last": len(ct) - 1}[where]
    bad[pos] ^= 0x04
    Kb, tr = O.decaps(p, sk, bad, trace=True)
    assert not tr["eq"]
    z = bytes(sk[8 * p.n:8 * p.n + 32])
    ch = [bytes(bad[i:i + O.TREE_CHUNK]) for i in range(0, len(bad), O.TREE_CHUNK)]
    hc = hashlib.sha3_256(b"".join(hashlib.sha3_256(y).digest() for y in ch)).digest()
    assert bytes(Kb) == hashlib.sha3_256(z + hc).digest()
    assert not np.array_equal(Kb, K)
    _, tr_ok = O.decaps(p, sk, ct, trace=True)
    assert tr_ok["eq"]


@pytest.mark.parametrize("name", ["P640", "P1344"])
def test_decode_closed_form(name):
    """Dec(x) = round(x / 2^(D-B)) mod 2^B with ties up (Alg. 3 generalised
    to B bits): a ciphertext with B' = 0 decrypts C directly."""
    p = _params(name)
    D, Bb = p.logq, p.B
    pk, sk = O.keygen(p, bytes(master_seeds(1, 5)[0]))
    r = np.random.default_rng(9)
    half = 1 << (D - Bb - 1)
    for trial in range(4):
        sym = r.integers(0, 1 << Bb, size=64)
        err = r.integers(-half, half, size=64)           # strictly inside
        if trial == 3:
            err[:8] = half                                # exact ties round up
            err[8:16] = -half
        C = (sym * (1 << (D - Bb)) + err) % (1 << D)
        ct = np.zeros(O.sizes(p)[2], np.uint8)
        ct[16 * p.n:] = np.frombuffer(C.astype("<u2").tobytes(), np.uint8)
        _, tr = O.decaps(p, sk, ct, trace=True)
        assert np.array_equal(tr["M"].reshape(-1).astype(np.int64), C)
        expect = sym.copy()
        if trial == 3:
            expect[:8] = (sym[:8] + 1) % (1 << Bb)
        bits = np.unpackbits(np.frombuffer(tr["mu"], np.uint8), bitorder="little")
        got = np.array([sum(int(bits[i * Bb + u]) << u for u in range(Bb)) for i in range(64)])
        assert np.array_equal(got, expect)


def test_decryption_noise_variance():
    """M - Enc(mu) = S'E - E'S + E'' (from Alg. 1-3): each coefficient has
    variance 2 n s^4 + s^2 with s^2 the sampler's variance."""
    p = _params("P640")
    T = O.cdf_table(p.sigma, p.clip)
    vals = np.array([O.sample(w, T, p.clip) for w in range(65536)], dtype=np.float64)
    s2 = (vals ** 2).mean()
    expect = 2 * p.n * s2 * s2 + s2
    pk, sk = O.keygen(p, bytes(master_seeds(1, 6)[0]))
    D, Bb = p.logq, p.B
    q = 1 << D
    noise = []
    for c in coins(40, seed=6):
        ct, K, tre = O.encaps(p, pk, bytes(c), trace=True)
        _, trd = O.decaps(p, sk, ct, trace=True)
        bits = np.unpackbits(np.frombuffer(tre["mu"], np.uint8), bitorder="little")
        sym = np.array([sum(int(bits[i * Bb + u]) << u for u in range(Bb)) for i in range(64)])
        d = (trd["M"].reshape(-1).astype(np.int64) - sym * (1 << (D - Bb))) % q
        noise.append(np.where(d >= q // 2, d - q, d))
    noise = np.concatenate(noise).astype(np.float64)
    assert abs(noise.mean()) < 4 * np.sqrt(expect / noise.size) * 3
    assert abs(noise.var() / expect - 1.0) < 0.15


def test_invalid_parameters_rejected():
    assert not O.check_params(O.Params(n=12, logq=16, B=2, clip=10, sigma=2.3))
    assert not O.check_params(O.Params(n=64, logq=16, B=5, clip=10, sigma=2.3))
    assert not O.check_params(O.Params(n=64, logq=3, B=3, clip=10, sigma=2.3))
    # a clip far in the tail gives a non-increasing table
    assert not O.check_params(O.Params(n=64, logq=16, B=2, clip=15, sigma=0.6))
    for name in PRESETS:
        assert O.check_params(_params(name))
