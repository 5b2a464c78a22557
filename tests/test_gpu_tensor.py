"""GPU parity of the batched tensor-core path (stacked S' times [A | B] as an
exact two-limb bf16 tcgen05 GEMM) against the CPU oracle.

Sizes span several 128-row tiles and 64/128-column tiles with ragged M, N
and K tails; the worst-case limb magnitudes check that the fp32 accumulation
stays exact.  All comparisons are bit-exact."""
import numpy as np
import pytest
import torch

from gpu_util import (O, PRESETS, as_u16, cfg_key, coins, dev, host, lwe, master_seeds,
                      oracle_keys, params)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _sa_ctx(n, logq, items, bn=128, clip=12):
    p = lwe.Params(n=n, logq=logq, B=2, clip=clip, sigma=2.8 if clip == 12 else 2.3)
    ctx = lwe.Ctx(p, max_batch=items)
    ctx.set_path(lwe.PATH_TENSOR)
    ctx.set_option(lwe.OPT_GEMM_PAIR, 0)  # the single-CTA kernel (the pair kernel: test_gpu_pair)
    ctx.set_option(lwe.OPT_GEMM_BN, bn)
    return ctx


@pytest.mark.parametrize("n,logq,items", [(64, 16, 1), (80, 15, 17), (208, 16, 16),
                                          (976, 16, 37), (1344, 16, 20)])
@pytest.mark.parametrize("stored", [True, False])
@pytest.mark.parametrize("bn", [128, 64])
def test_matmul_modq_SA_tensor_matches_oracle(n, logq, items, stored, bn):
    k = 8 * items
    r = np.random.default_rng(n * items + bn)
    seed = r.integers(0, 256, 16, dtype=np.uint8)
    A_o = O.expand_A(bytes(seed), n, logq)
    S = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    E = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    ctx = _sa_ctx(n, logq, items, bn)
    out = torch.empty((k, n), dtype=torch.int16, device="cuda")
    A = dev(A_o.view(np.int16)) if stored else None
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, logq, A=A, seedA=dev(seed), E=dev(E), ctx=ctx)
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, E, logq))
    assert ctx.device_error() == 0


@pytest.mark.parametrize("clip", [10, 12])
def test_tensor_exact_at_worst_case_limbs(clip):
    """A = 0x8080 splits into the extreme limbs (-128, -127); S = +c makes
    every partial sum as large as the accumulator ever sees."""
    n, logq, items = 976, 16, 16
    k = 8 * items
    A_o = np.full((n, n), 0x8080, dtype=np.uint16)
    S = np.full((k, n), clip, dtype=np.int8)
    S[1::2] = -clip
    ctx = _sa_ctx(n, logq, items, clip=clip)
    out = torch.empty((k, n), dtype=torch.int16, device="cuda")
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, logq, A=dev(A_o.view(np.int16)), ctx=ctx)
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, None, logq))


@pytest.mark.parametrize("name,count", [("P640", 21), ("P976", 37), ("P1344", 19)])
@pytest.mark.parametrize("stored", [True, False])
@pytest.mark.parametrize("pair", [1, 0])
def test_kem_tensor_path_matches_oracle(name, count, stored, pair):
    cfg = PRESETS[name]
    p, po = params(name)
    pk_o, sk_o, A_o, ms = oracle_keys(cfg_key(cfg), 21)
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(lwe.PATH_TENSOR)
    ctx.set_option(lwe.OPT_GEMM_PAIR, pair)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda") if stored else None
    ctx.keygen(dev(ms[None, :]), pk, sk, A_out=A)
    cs = coins(count, seed=31)
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps(pk, dev(cs), ct, K, A=A)
    K2 = torch.empty_like(K)
    ctx.decaps(sk, ct, K2, A=A)
    bad = ct.clone()
    bad[::3, 7] ^= 2
    bad[1::3, -3] ^= 1
    Kb = torch.empty_like(K)
    ctx.decaps(sk, bad, Kb, A=A)
    ct_h, K_h, K2_h, Kb_h, bad_h = host(ct), host(K), host(K2), host(Kb), host(bad)
    for i in range(count):
        ct_o, K_o = O.encaps(po, pk_o, bytes(cs[i]), A=A_o)
        assert np.array_equal(ct_h[i], ct_o), i
        assert np.array_equal(K_h[i], K_o), i
        assert np.array_equal(K2_h[i], K_o), i
    for i in list(range(0, count, 3)) + list(range(1, count, 3))[:3]:
        assert np.array_equal(Kb_h[i], O.decaps(po, sk_o, bad_h[i], A=A_o)), i
    assert ctx.device_error() == 0


def test_batched_4096_tensor_equals_skinny_and_oracle():
    """The benchmarked workload: one P976 key, 4096 encapsulations then the
    4096 decapsulations, on the tensor path; every item equals the CUDA-core
    path's and the oracle's (all 4096 ciphertexts and both key sets, the
    oracle's batch run on every host core)."""
    name, count = "P976", 4096
    cfg = PRESETS[name]
    p, po = params(name)
    pk_o, sk_o, A_o, ms = oracle_keys(cfg_key(cfg), 21)
    ctx = lwe.Ctx(p, max_batch=count)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
    ctx.keygen(dev(ms[None, :]), pk, sk, A_out=A)
    cs = coins(count, seed=4096)
    res = {}
    for path in (lwe.PATH_TENSOR, lwe.PATH_SKINNY):
        ctx.set_path(path)
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, dev(cs), ct, K, A=A)
        K2 = torch.empty_like(K)
        ctx.decaps(sk, ct, K2, A=A)
        res[path] = (host(ct), host(K), host(K2))
    ct_t, K_t, K2_t = res[lwe.PATH_TENSOR]
    ct_s, K_s, K2_s = res[lwe.PATH_SKINNY]
    assert np.array_equal(ct_t, ct_s)
    assert np.array_equal(K_t, K_s)
    assert np.array_equal(K2_t, K_t)
    assert np.array_equal(K2_s, K_s)
    ct_o, K_o = O.encaps_batch(po, pk_o, cs, A=A_o, nthreads=O.max_threads())
    bad = np.nonzero((ct_t != ct_o).any(axis=1))[0]
    assert bad.size == 0, "ciphertexts differ from the oracle at %s" % bad[:8]
    assert np.array_equal(K_t, K_o)
    K2_o = O.decaps_batch(po, sk_o, ct_t, A=A_o, nthreads=O.max_threads())
    assert np.array_equal(K2_t, K2_o)
    assert ctx.device_error() == 0


@pytest.mark.parametrize("path", [lwe.PATH_TENSOR, lwe.PATH_SKINNY])
def test_bound_key_gives_the_same_results(path):
    """lwe_ctx_bind_key makes H(pk) and the limbs once; bound calls equal
    unbound ones, also after a tensor-path call for another key has
    overwritten the limb workspace, and after unbinding."""
    name, count = "P976", 80
    p, po = params(name)
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(path)
    keys = []
    for s in (41, 42):
        pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
        A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
        ctx.keygen(dev(master_seeds(1, seed=s)), pk, sk, A_out=A)
        keys.append((pk, sk, A))
    (pk, sk, A), (pk2, sk2, A2) = keys
    cs = dev(coins(count, seed=43))

    def run(pk, sk, A):
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, cs, ct, K, A=A)
        K2 = torch.empty_like(K)
        ctx.decaps(sk, ct, K2, A=A)
        return host(ct), host(K), host(K2)

    ref = run(pk, sk, A)
    ref2 = run(pk2, sk2, A2)
    ctx.bind_key(pk, sk, A)
    # bound, another key in between (overwrites the limbs), bound again
    for keyset, want in (((pk, sk, A), ref), ((pk2, sk2, A2), ref2), ((pk, sk, A), ref)):
        for x, y in zip(run(*keyset), want):
            assert np.array_equal(x, y)
    ctx.bind_key(None, sk, None)  # sk only, stored A not bound: regenerated A
    c_fused = run(pk, sk, None)
    ctx.bind_key(None)
    d_fused = run(pk, sk, None)
    for x, y in zip(c_fused, d_fused):
        assert np.array_equal(x, y)
    for x, y in zip(c_fused, ref):
        assert np.array_equal(x, y)
    assert ctx.device_error() == 0


def test_graph_replay_equals_direct_calls():
    """The captured Encaps+Decaps step, replayed with new coins, gives what
    the direct calls give."""
    from paper_2606_01211_gb300 import batch
    kem = batch.BatchedKem("P976", 96, seed=9)
    kem.capture()
    for s in (1, 2):
        cs = dev(coins(96, seed=900 + s))
        kem.replay(cs)
        torch.cuda.synchronize()
        ct_g, K_g, K2_g = kem.ct.clone(), kem.K.clone(), kem.K2.clone()
        ct = kem.ctx.empty_ct(96)
        K = torch.empty((96, 32), dtype=torch.uint8, device="cuda")
        kem.ctx.encaps(kem.pk, cs, ct, K, A=kem.A)
        assert torch.equal(ct, ct_g) and torch.equal(K, K_g) and torch.equal(K2_g, K_g)
    kem.close()


def test_autotune_returns_a_valid_choice():
    from paper_2606_01211_gb300 import batch
    res = batch.autotune("P640", 256, cache=None)
    assert res["gemm_bn"] in (64, 128) and res["gemm_pair"] in (0, 1)
    assert 16 <= res["tensor_min"] <= 257
