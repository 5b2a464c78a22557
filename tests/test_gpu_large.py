"""Large parameter sets (n = 16384 and 32768, A of 0.5 / 2 GiB) and the K-split
tensor path, checked against the oracle on sampled outputs.

At these sizes the oracle cannot recompute whole products in seconds, so each
test recomputes, with oracle primitives only, what a sampled output depends
on: the seeds and noise streams (SHA3-256, AES-CTR sampler), a row of A for a
sampled row of B = A S + E (Alg. 1), a column of A for a sampled column of
B' = S' A + E' (Alg. 2), the whole V = S' B + E'' and C, and the keys of
Alg. 4-5 from the tree hash of the produced ciphertext.  Stored and
regenerated A, and the CUDA-core and tensor-core paths, must agree on every
item bit for bit.
"""
import numpy as np
import pytest
import torch

from gpu_util import O, PRESETS, as_u16, coins, dev, host, lwe, master_seeds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _A_row(seedA, n, logq, i):
    ks = O.ctr_blocks(seedA, 0, i * (n // 8), n // 8)
    return (np.frombuffer(ks, dtype="<u2") & ((1 << logq) - 1)).astype(np.uint16)


def _A_col(seedA, n, logq, j):
    col = np.zeros(n, np.uint16)
    for i in range(n):
        blk = O.ctr_blocks(seedA, 0, i * (n // 8) + j // 8, 1)
        col[i] = (int.from_bytes(blk[2 * (j % 8):2 * (j % 8) + 2], "little")) & ((1 << logq) - 1)
    return col


def _check_keygen(po, ms, pk_h, sk_h, rows):
    n, logq = po.n, po.logq
    T = O.cdf_table(po.sigma, po.clip)
    seedA = O.sha3_256(b"\x41" + ms)[:16]
    seedSE = O.sha3_256(b"\x53" + ms)[:16]
    assert bytes(pk_h[:16]) == seedA
    St = O.noise(seedSE, 1, T, po.clip, 8 * n).reshape(8, n)
    assert np.array_equal(sk_h[:8 * n].view(np.int8).reshape(8, n), St)
    assert bytes(sk_h[8 * n:8 * n + 32]) == O.sha3_256(b"\x5a" + ms)
    assert bytes(sk_h[8 * n + 32:8 * n + 64]) == O.htree(bytes(pk_h))
    assert np.array_equal(sk_h[8 * n + 64:], pk_h)
    E = O.noise(seedSE, 2, T, po.clip, 8 * (max(rows) + 1)).reshape(-1, 8)
    B = np.frombuffer(pk_h[16:].tobytes(), dtype="<u2").reshape(n, 8)
    for i in rows:
        Ai = _A_row(seedA, n, logq, i)
        ref = O.mul_SA(St, Ai.reshape(n, 1), E[i].reshape(8, 1), logq).reshape(8)
        assert np.array_equal(B[i], ref), i
    return seedA, St


def _check_encaps(po, pk_h, seedA, c, ct_h, K_h, cols):
    n, logq, Bb = po.n, po.logq, po.B
    T = O.cdf_table(po.sigma, po.clip)
    mub = O.sizes(po)[3]
    mu = O.sha3_256(b"\x4d" + c)[:mub]
    pkh = O.htree(bytes(pk_h))
    kp = O.sha3_256(pkh + mu)
    seed = O.sha3_256(b"\x01" + pkh + mu)[:16]
    Sp = O.noise(seed, 3, T, po.clip, 8 * n).reshape(8, n)
    Ep = O.noise(seed, 4, T, po.clip, 8 * n).reshape(8, n)
    Epp = O.noise(seed, 5, T, po.clip, 64).reshape(8, 8)
    Bp = np.frombuffer(ct_h[:16 * n].tobytes(), dtype="<u2").reshape(8, n)
    for j in cols:
        col = _A_col(seedA, n, logq, j)
        ref = O.mul_SA(Sp, col.reshape(n, 1), Ep[:, j:j + 1].copy(), logq).reshape(8)
        assert np.array_equal(Bp[:, j], ref), j
    Bm = np.frombuffer(pk_h[16:].tobytes(), dtype="<u2").reshape(n, 8)
    V = O.mul_SA(Sp, Bm, Epp, logq).astype(np.int64)
    bits = np.unpackbits(np.frombuffer(mu, np.uint8), bitorder="little")
    sym = np.array([sum(int(bits[i * Bb + u]) << u for u in range(Bb)) for i in range(64)]).reshape(8, 8)
    C = (V + sym * (1 << (logq - Bb))) % (1 << logq)
    assert np.array_equal(np.frombuffer(ct_h[16 * n:].tobytes(), dtype="<u2").reshape(8, 8), C)
    assert bytes(K_h) == O.sha3_256(kp + O.htree(bytes(ct_h)))


@pytest.mark.parametrize("name", ["P16384", "P32768"])
def test_large_kem_stored_and_fused_sampled_against_oracle(name):
    cfg = PRESETS[name]
    p, po = lwe.Params(**cfg), O.Params(**cfg)
    n = p.n
    ms = master_seeds(1, seed=16)
    cs = coins(2, seed=16)
    out = {}
    for stored in (True, False):
        ctx = lwe.Ctx(p, max_batch=2)
        pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
        A = torch.empty((n, n), dtype=torch.int16, device="cuda") if stored else None
        ctx.keygen(dev(ms), pk, sk, A_out=A)
        ct = ctx.empty_ct(2)
        K = torch.empty((2, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, dev(cs), ct, K, A=A)
        K2 = torch.empty_like(K)
        ctx.decaps(sk, ct, K2, A=A)
        bad = ct.clone()
        bad[1, 16 * n + 5] ^= 1
        Kb = torch.empty_like(K)
        ctx.decaps(sk, bad, Kb, A=A)
        out[stored] = [host(x) for x in (pk, sk, ct, K, K2, Kb, bad)]
        if stored:
            # spot rows of the stored A against the AES stream
            ah = torch.empty(n, dtype=torch.int16)
            ah.copy_(A[n - 3])
            out["Arow"] = ah.numpy().view(np.uint16)
        assert ctx.device_error() == 0
        del A
        ctx.close()
        torch.cuda.empty_cache()
    for a, b in zip(out[True], out[False]):
        assert np.array_equal(a, b)
    pk_h, sk_h, ct_h, K_h, K2_h, Kb_h, bad_h = out[True]
    seedA, St = _check_keygen(po, bytes(ms[0]), pk_h[0], sk_h[0], rows=[0, 1, n // 2, n - 1])
    assert np.array_equal(out["Arow"], _A_row(seedA, n, po.logq, n - 3))
    _check_encaps(po, pk_h[0], seedA, bytes(cs[0]), ct_h[0], K_h[0], cols=[0, n - 1])
    assert np.array_equal(K2_h, K_h)
    z = bytes(sk_h[0][8 * n:8 * n + 32])
    assert bytes(Kb_h[1]) == O.sha3_256(z + O.htree(bytes(bad_h[1])))
    assert np.array_equal(Kb_h[0], K_h[0])


def test_large_batched_tensor_ksplit_equals_cuda_cores_and_oracle():
    """P16384 with 64 encapsulations: the tensor path runs as two K passes."""
    cfg = PRESETS["P16384"]
    p, po = lwe.Params(**cfg), O.Params(**cfg)
    n, count = p.n, 64
    ctx = lwe.Ctx(p, max_batch=count)
    ms = master_seeds(1, seed=17)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((n, n), dtype=torch.int16, device="cuda")
    ctx.keygen(dev(ms), pk, sk, A_out=A)
    cs = coins(count, seed=17)
    res = {}
    for path in (lwe.PATH_TENSOR, lwe.PATH_SKINNY):
        ctx.set_path(path)
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, dev(cs), ct, K, A=A)
        K2 = torch.empty_like(K)
        ctx.decaps(sk, ct, K2, A=A)
        res[path] = (host(ct), host(K), host(K2))
    assert np.array_equal(res[lwe.PATH_TENSOR][0], res[lwe.PATH_SKINNY][0])
    assert np.array_equal(res[lwe.PATH_TENSOR][1], res[lwe.PATH_SKINNY][1])
    assert np.array_equal(res[lwe.PATH_TENSOR][2], res[lwe.PATH_TENSOR][1])
    pk_h = host(pk)[0]
    seedA = O.sha3_256(b"\x41" + bytes(ms[0]))[:16]
    ct_h, K_h, _ = res[lwe.PATH_TENSOR]
    _check_encaps(po, pk_h, seedA, bytes(cs[63]), ct_h[63], K_h[63], cols=[8191, 10880, n - 1])
    assert ctx.device_error() == 0


@pytest.mark.parametrize("kchunk", [64, 256, 512])
def test_ksplit_passes_match_oracle_at_n976(kchunk):
    """Forcing small K passes at n = 976 exercises the running-sum buffer
    (first / middle / last pass) against the full oracle."""
    cfg = PRESETS["P976"]
    p, po = lwe.Params(**cfg), O.Params(**cfg)
    n, count = p.n, 19
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(lwe.PATH_TENSOR)
    ctx.set_option(lwe.OPT_GEMM_KCHUNK, kchunk)
    ms = master_seeds(1, seed=18)
    pk_o, sk_o, A_o = O.keygen(po, bytes(ms[0]), want_A=True)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    ctx.keygen(dev(ms), pk, sk)
    cs = coins(count, seed=18)
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps(pk, dev(cs), ct, K)
    K2 = torch.empty_like(K)
    ctx.decaps(sk, ct, K2)
    ct_h, K_h, K2_h = host(ct), host(K), host(K2)
    for i in range(count):
        ct_o, K_o = O.encaps(po, pk_o, bytes(cs[i]), A=A_o)
        assert np.array_equal(ct_h[i], ct_o), i
        assert np.array_equal(K_h[i], K_o), i
    assert np.array_equal(K2_h, K_h)
    # the standalone product with the same passes
    r = np.random.default_rng(kchunk)
    S = r.integers(-10, 11, size=(8 * count, n), dtype=np.int8)
    out = torch.empty((8 * count, n), dtype=torch.int16, device="cuda")
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, 16, A=dev(A_o.view(np.int16)), ctx=ctx)
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, None, 16))
    with pytest.raises(lwe.LweError):
        ctx.set_option(lwe.OPT_GEMM_KCHUNK, 100)
