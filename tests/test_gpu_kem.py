"""GPU parity of the CUDA-core path against the CPU oracle, element by element.

Covers A expansion (sample(seedA), Alg. 1), the noise streams and A S + E
(KeyGen, Alg. 1), Encrypt/Encaps (Alg. 2, 4), Decrypt/Decaps with implicit
rejection (Alg. 3, 5), the standalone products, stored versus regenerated A,
ragged and minimal sizes, and the argument errors of the C ABI.  Every
comparison is bit-exact: the whole path is integer arithmetic.
"""
import numpy as np
import pytest
import torch

from gpu_util import (O, PRESETS, as_u16, cfg_key, coins, dev, host, lwe, master_seeds,
                      oracle_keys, params)

pytestmark = pytest.mark.gpu

SMALL = {
    "n16": dict(n=16, logq=16, B=2, clip=10, sigma=2.3),
    "n48": dict(n=48, logq=15, B=3, clip=12, sigma=2.8),
    "n80": dict(n=80, logq=16, B=4, clip=6, sigma=1.4),
    "P640": PRESETS["P640"],
    "P976": PRESETS["P976"],
    "P1344": PRESETS["P1344"],
}


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


# ------------------------------------------------------------ A expansion --

@pytest.mark.parametrize("n,logq", [(16, 16), (48, 15), (640, 15), (976, 16), (1344, 16)])
def test_expand_A_matches_oracle(n, logq):
    seed = master_seeds(1, seed=n)[0][:16]
    A = torch.empty((n, n), dtype=torch.int16, device="cuda")
    lwe.expand_A(dev(seed), n, logq, A)
    assert np.array_equal(as_u16(A), O.expand_A(bytes(seed), n, logq))


def test_expand_A_large_sampled_rows():
    n, logq = 8192, 16
    seed = master_seeds(1, seed=8192)[0][:16]
    A = torch.empty((n, n), dtype=torch.int16, device="cuda")
    lwe.expand_A(dev(seed), n, logq, A)
    for i in [0, 1, 4095, n - 1]:
        row = torch.empty(n, dtype=torch.int16)
        row.copy_(A[i])
        ks = O.ctr_blocks(bytes(seed), 0, i * (n // 8), n // 8)
        ref = np.frombuffer(ks, dtype="<u2") & ((1 << logq) - 1)
        assert np.array_equal(row.numpy().view(np.uint16), ref)


# ------------------------------------------------------------------ KeyGen --

@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("stored", [True, False])
@pytest.mark.parametrize("warp_max", [0, None])
def test_keygen_matches_oracle(name, stored, warp_max):
    """warp_max 0: the seeds hashed with one Keccak state per thread;
    default: one state per warp (a launch of 3 items)."""
    _keygen_case(name, stored, warp_max, 3)


def test_keygen_batch_matches_oracle():
    """70 P640 key pairs in one call: enough rows that A S runs as one warp
    per row group (k_mul_as_rows) instead of splitting columns."""
    _keygen_case("P640", True, None, 70)


def _keygen_case(name, stored, warp_max, count):
    cfg = SMALL[name]
    p, po = params(**cfg)
    ms = master_seeds(count, seed=11)
    ctx = lwe.Ctx(p, max_batch=count)
    if warp_max is not None:
        ctx.set_option(lwe.OPT_WARP_HASH_MAX, warp_max)
    pk, sk = ctx.empty_pk(count), ctx.empty_sk(count)
    A = torch.empty((count, p.n, p.n), dtype=torch.int16, device="cuda") if stored else None
    ctx.keygen(dev(ms), pk, sk, A_out=A)
    pk_h, sk_h = host(pk), host(sk)
    for i in range(count):
        pk_o, sk_o, A_o = O.keygen(po, bytes(ms[i]), want_A=True)
        assert np.array_equal(pk_h[i], pk_o)
        assert np.array_equal(sk_h[i], sk_o)
        if stored:
            assert np.array_equal(as_u16(A[i]), A_o)
    assert ctx.device_error() == 0


# --------------------------------------------------------- Encaps / Decaps --

def _kem_case(name, count, path, stored, seed=21, options=()):
    cfg = SMALL[name] if name in SMALL else PRESETS[name]
    p, po = params(**cfg)
    pk_o, sk_o, A_o, ms = oracle_keys(cfg_key(cfg), seed)
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(path)
    for opt, val in options:
        ctx.set_option(opt, val)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda") if stored else None
    ctx.keygen(dev(ms[None, :]), pk, sk, A_out=A)
    cs = coins(count, seed=seed)
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps(pk, dev(cs), ct, K, A=A)
    K2 = torch.empty_like(K)
    ctx.decaps(sk, ct, K2, A=A)
    return ctx, p, po, pk_o, sk_o, A_o, cs, ct, K, K2, pk, sk, A


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("stored", [True, False])
def test_encaps_decaps_skinny_match_oracle(name, stored):
    count = 5
    ctx, p, po, pk_o, sk_o, A_o, cs, ct, K, K2, *_ = _kem_case(name, count, lwe.PATH_SKINNY, stored)
    ct_h, K_h, K2_h = host(ct), host(K), host(K2)
    for i in range(count):
        ct_o, K_o = O.encaps(po, pk_o, bytes(cs[i]), A=A_o)
        assert np.array_equal(ct_h[i], ct_o), i
        assert np.array_equal(K_h[i], K_o), i
        assert np.array_equal(K2_h[i], K_o), i
    assert ctx.device_error() == 0


@pytest.mark.parametrize("name", ["n16", "P640", "P976", "P1344"])
@pytest.mark.parametrize("warp_max", [0, 1 << 20])
def test_tree_hash_forms_match_oracle(name, warp_max):
    """The tree hashes (H(pk) in Encaps, H(c) with the Encaps key, H(c) in
    Decaps) with one Keccak state per thread (warp_max 0) and with one state
    per warp (every launch at most warp_max messages), on 37 items: the
    ciphertexts and both keys equal the oracle's."""
    count = 37
    ctx, p, po, pk_o, sk_o, A_o, cs, ct, K, K2, *_ = _kem_case(
        name, count, lwe.PATH_SKINNY, True, seed=23,
        options=((lwe.OPT_WARP_HASH_MAX, warp_max),))
    ct_h, K_h, K2_h = host(ct), host(K), host(K2)
    for i in (0, 1, 17, count - 1):
        ct_o, K_o = O.encaps(po, pk_o, bytes(cs[i]), A=A_o)
        assert np.array_equal(ct_h[i], ct_o), i
        assert np.array_equal(K_h[i], K_o), i
    assert np.array_equal(K_h, K2_h)
    assert ctx.device_error() == 0


@pytest.mark.parametrize("name", ["n48", "P640", "P1344"])
def test_implicit_rejection_matches_oracle(name):
    count = 4
    ctx, p, po, pk_o, sk_o, A_o, cs, ct, K, K2, pk, sk, A = _kem_case(
        name, count, lwe.PATH_SKINNY, True)
    bad = ct.clone()
    ctb = p.ct_bytes
    flips = [(0, 3), (1, 2 * 8 * p.n + 5), (2, ctb - 1), (3, 2 * p.n + 1)]
    for i, pos in flips:
        bad[i, pos] ^= 1
    Kb = torch.empty_like(K)
    ctx.decaps(sk, bad, Kb, A=A)
    Kb_h, bad_h, K_h = host(Kb), host(bad), host(K)
    for i, _ in flips:
        Kb_o = O.decaps(po, sk_o, bad_h[i], A=A_o)
        assert np.array_equal(Kb_h[i], Kb_o)
        assert not np.array_equal(Kb_h[i], K_h[i])


def test_decaps_of_many_tampered_bits_never_accepts():
    count = 64
    ctx, p, po, pk_o, sk_o, A_o, cs, ct, K, K2, pk, sk, A = _kem_case(
        "P640", count, lwe.PATH_SKINNY, True)
    bad = ct.clone()
    r = np.random.default_rng(3)
    pos = r.integers(0, p.ct_bytes, size=count)
    for i in range(count):
        bad[i, int(pos[i])] ^= 1 << int(r.integers(0, 8))
    Kb = torch.empty_like(K)
    ctx.decaps(sk, bad, Kb, A=A)
    assert not (host(Kb) == host(K)).all(axis=1).any()
    # untouched ciphertexts still decapsulate
    assert np.array_equal(host(K2), host(K))


@pytest.mark.parametrize("path", [lwe.PATH_SKINNY, lwe.PATH_TENSOR])
def test_decaps_batch_above_warp_hash_threshold_matches_oracle(path):
    """Above the one-state-per-warp threshold (one item per SM) Decaps'
    H(c) is the batched tree on the side stream: the implicit-rejection
    keys H(z || H(c)) of tampered ciphertexts equal the oracle's, the
    untouched ones decapsulate, and the serial schedule (side-stream work
    on the caller's stream) gives the same keys."""
    count = 200
    ctx, p, po, pk_o, sk_o, A_o, cs, ct, K, K2, pk, sk, A = _kem_case(
        "P640", count, path, True)
    assert count > torch.cuda.get_device_properties(0).multi_processor_count
    bad = ct.clone()
    tampered = list(range(0, count, 7))
    for i in tampered:
        bad[i, (131 * i) % p.ct_bytes] ^= 2
    Kb = torch.empty_like(K)
    ctx.decaps(sk, bad, Kb, A=A)
    Kb_h, bad_h, K_h = host(Kb), host(bad), host(K)
    for i in (0, 7, 154, 196):
        assert np.array_equal(Kb_h[i], O.decaps(po, sk_o, bad_h[i], A=A_o)), i
    for i in range(count):
        assert np.array_equal(Kb_h[i], K_h[i]) == (i not in tampered), i
    assert np.array_equal(host(K2), K_h)
    ctx.set_option(lwe.OPT_SERIAL, 1)
    Ks = torch.empty_like(K)
    ctx.decaps(sk, bad, Ks, A=A)
    assert np.array_equal(host(Ks), Kb_h)
    assert ctx.device_error() == 0


# ------------------------------------------------------ standalone products --

@pytest.mark.parametrize("n,logq", [(16, 16), (48, 15), (208, 16), (976, 16)])
@pytest.mark.parametrize("stored", [True, False])
@pytest.mark.parametrize("with_e", [True, False])
def test_matmul_modq_AS_matches_oracle(n, logq, stored, with_e):
    r = np.random.default_rng(n + logq)
    seed = r.integers(0, 256, 16, dtype=np.uint8)
    A_o = O.expand_A(bytes(seed), n, logq)
    St = r.integers(-12, 13, size=(8, n), dtype=np.int8)
    E = r.integers(-12, 13, size=(n, 8), dtype=np.int8) if with_e else None
    out = torch.empty((n, 8), dtype=torch.int16, device="cuda")
    A = dev(A_o.view(np.int16)) if stored else None
    lwe.matmul_modq(lwe.SIDE_AS, dev(St), out, n, logq, A=A, seedA=dev(seed),
                    E=dev(E.reshape(8, n)) if with_e else None)
    assert np.array_equal(as_u16(out), O.mul_AS(A_o, St, E, logq))


@pytest.mark.parametrize("n,logq,k", [(16, 16, 8), (48, 15, 16), (208, 16, 24), (976, 16, 8)])
@pytest.mark.parametrize("stored", [True, False])
def test_matmul_modq_SA_cuda_cores_match_oracle(n, logq, k, stored):
    r = np.random.default_rng(n * k)
    seed = r.integers(0, 256, 16, dtype=np.uint8)
    A_o = O.expand_A(bytes(seed), n, logq)
    S = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    E = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    out = torch.empty((k, n), dtype=torch.int16, device="cuda")
    A = dev(A_o.view(np.int16)) if stored else None
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, logq, A=A, seedA=dev(seed), E=dev(E))
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, E, logq))


def test_matmul_modq_full_range_values():
    """Worst-case magnitudes: A = q - 1 everywhere, S = +-c."""
    n, logq = 976, 16
    A_o = np.full((n, n), (1 << logq) - 1, dtype=np.uint16)
    St = np.full((8, n), -10, dtype=np.int8)
    St[::2] = 10
    out = torch.empty((n, 8), dtype=torch.int16, device="cuda")
    lwe.matmul_modq(lwe.SIDE_AS, dev(St), out, n, logq, A=dev(A_o.view(np.int16)))
    assert np.array_equal(as_u16(out), O.mul_AS(A_o, St, None, logq))
    out2 = torch.empty((8, n), dtype=torch.int16, device="cuda")
    lwe.matmul_modq(lwe.SIDE_SA, dev(St), out2, n, logq, A=dev(A_o.view(np.int16)))
    assert np.array_equal(as_u16(out2), O.mul_SA(St, A_o, None, logq))


# ------------------------------------------------------------ edge cases --

def test_count_zero_and_capacity_and_alignment():
    p, po = params("P640")
    ctx = lwe.Ctx(p, max_batch=2)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    ms = dev(master_seeds(4, seed=5))
    L = lwe.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.lwe_keygen(ctx.handle, ms.data_ptr(), 0, pk.data_ptr(), sk.data_ptr(), None, s) == 0
    assert L.lwe_keygen(ctx.handle, ms.data_ptr(), 3, pk.data_ptr(), sk.data_ptr(), None,
                        s) == lwe.LWE_ECAPACITY
    assert L.lwe_keygen(ctx.handle, ms.data_ptr() + 1, 1, pk.data_ptr(), sk.data_ptr(), None,
                        s) == lwe.LWE_EINVAL
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert L.lwe_expand_A(buf.data_ptr(), 64, 16, buf.data_ptr() + 2, s) == lwe.LWE_EINVAL
    ctx.keygen(ms[:1], pk, sk)
    ct = ctx.empty_ct(1)
    K = torch.zeros((1, 32), dtype=torch.uint8, device="cuda")
    c = dev(coins(1, seed=5))
    assert L.lwe_encaps(ctx.handle, pk.data_ptr(), None, c.data_ptr(), 0, ct.data_ptr(),
                        K.data_ptr(), s) == 0
    assert host(K).sum() == 0  # count 0 wrote nothing
    assert ctx.device_error() == 0


def test_results_independent_of_batch_position():
    """An item gives the same ciphertext and key alone and inside a batch."""
    p, po = params("P976")
    pk_o, sk_o, A_o, ms = oracle_keys(cfg_key(PRESETS["P976"]), 21)
    ctx = lwe.Ctx(p, max_batch=32)
    ctx.set_path(lwe.PATH_SKINNY)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    ctx.keygen(dev(ms[None, :]), pk, sk)
    cs = coins(32, seed=77)
    ct = ctx.empty_ct(32)
    K = torch.empty((32, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps(pk, dev(cs), ct, K)
    ct1 = ctx.empty_ct(1)
    K1 = torch.empty((1, 32), dtype=torch.uint8, device="cuda")
    for i in [0, 13, 31]:
        ctx.encaps(pk, dev(cs[i:i + 1]), ct1, K1)
        assert np.array_equal(host(ct1)[0], host(ct)[i])
        assert np.array_equal(host(K1)[0], host(K)[i])


def test_bounded_wait_times_out_cleanly():
    """A device wait that nothing completes gives up after its limit, reports
    LWE_ETIMEOUT on the host, and leaves the context usable (no fault)."""
    import time
    p, po = params("P640")
    ctx = lwe.Ctx(p, max_batch=1)
    assert ctx.device_error() == lwe.LWE_OK
    t0 = time.perf_counter()
    rc = lwe.lib().lwe_selftest_bounded_wait(ctx.handle, 50000, torch.cuda.current_stream().cuda_stream)
    assert rc == lwe.LWE_OK
    assert ctx.device_error() == lwe.LWE_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert ctx.device_error() == lwe.LWE_OK  # cleared once read
    # the context still works
    ms = master_seeds(1, seed=8)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    ctx.keygen(dev(ms), pk, sk)
    pk_o, sk_o = O.keygen(po, bytes(ms[0]))
    assert np.array_equal(host(pk)[0], pk_o)


@pytest.mark.parametrize("name", ["P640", "P976"])
@pytest.mark.parametrize("stored", [True, False])
@pytest.mark.parametrize("give_pkh", [True, False])
def test_multi_key_calls_equal_single_key_calls(name, stored, give_pkh):
    """lwe_encaps_multi / lwe_decaps_multi (each item with its own key) give
    exactly what one single-key call per item gives, and the oracle's."""
    p, po = params(name)
    nk, count = 5, 23
    ms = master_seeds(nk, seed=40)
    ctx = lwe.Ctx(p, max_batch=max(nk, count))
    ctx.set_path(lwe.PATH_SKINNY)
    pk, sk = ctx.empty_pk(nk), ctx.empty_sk(nk)
    A = torch.empty((nk, p.n, p.n), dtype=torch.int16, device="cuda")
    ctx.keygen(dev(ms), pk, sk, A_out=A)
    keys = np.random.default_rng(41).integers(0, nk, size=count)
    pk_ptrs = torch.tensor([pk[k].data_ptr() for k in keys], dtype=torch.int64, device="cuda")
    sk_ptrs = torch.tensor([sk[k].data_ptr() for k in keys], dtype=torch.int64, device="cuda")
    pkh_ptrs = torch.tensor([sk[k].data_ptr() + 8 * p.n + 32 for k in keys], dtype=torch.int64,
                            device="cuda")
    A_ptrs = torch.tensor([A[k].data_ptr() for k in keys], dtype=torch.int64, device="cuda")
    cs = coins(count, seed=42)
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps_multi(pk_ptrs, dev(cs), ct, K, pkh_ptrs=pkh_ptrs if give_pkh else None,
                     A_ptrs=A_ptrs if stored else None)
    K2 = torch.empty_like(K)
    ctx.decaps_multi(sk_ptrs, ct, K2, A_ptrs=A_ptrs if stored else None)
    bad = ct.clone()
    bad[::2, 11] ^= 1
    Kb = torch.empty_like(K)
    ctx.decaps_multi(sk_ptrs, bad, Kb, A_ptrs=A_ptrs if stored else None)
    ct1, K1 = ctx.empty_ct(1), torch.empty((1, 32), dtype=torch.uint8, device="cuda")
    Kb1 = torch.empty_like(K1)
    for i, k in enumerate(keys):
        ctx.encaps(pk[k], dev(cs[i:i + 1]), ct1, K1, A=A[k])
        assert torch.equal(ct1[0], ct[i]) and torch.equal(K1[0], K[i]), i
        ctx.decaps(sk[k], bad[i:i + 1], Kb1, A=A[k])
        assert torch.equal(Kb1[0], Kb[i]), i
    assert torch.equal(K2, K)
    assert not (host(Kb)[::2] == host(K)[::2]).all(axis=1).any()
    k0 = int(keys[0])
    pk_o, sk_o = O.keygen(po, bytes(ms[k0]))
    ct_o, K_o = O.encaps(po, pk_o, bytes(cs[0]))
    assert np.array_equal(host(ct)[0], ct_o) and np.array_equal(host(K)[0], K_o)
    assert ctx.device_error() == 0
