"""GPU parity of the CTA-pair tensor-core product (tcgen05 cta_group::2:
two SMs share one 256-row tile, each loading its own rows of S' and one limb
tile) against the CPU oracle, bit-exact.

Row counts cover a tail tile whose second CTA has some rows, one whose second
CTA has none (it then loads no S'), several tiles per cluster, the ragged
column tile of [A | B] and the K-split passes."""
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


def _pair_ctx(p, items):
    ctx = lwe.Ctx(p, max_batch=items)
    ctx.set_path(lwe.PATH_TENSOR)
    ctx.set_option(lwe.OPT_GEMM_PAIR, 1)
    return ctx


@pytest.mark.parametrize("n,logq,items", [(64, 16, 1), (80, 15, 16), (208, 16, 17),
                                          (976, 16, 33), (976, 16, 64), (1344, 16, 20)])
@pytest.mark.parametrize("stored", [True, False])
def test_pair_matmul_SA_matches_oracle(n, logq, items, stored):
    k = 8 * items
    r = np.random.default_rng(7 * n + items)
    seed = r.integers(0, 256, 16, dtype=np.uint8)
    A_o = O.expand_A(bytes(seed), n, logq)
    S = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    E = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    ctx = _pair_ctx(lwe.Params(n=n, logq=logq, B=2, clip=12, sigma=2.8), items)
    out = torch.empty((k, n), dtype=torch.int16, device="cuda")
    A = dev(A_o.view(np.int16)) if stored else None
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, logq, A=A, seedA=dev(seed), E=dev(E), ctx=ctx)
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, E, logq))
    assert ctx.device_error() == 0


@pytest.mark.parametrize("n,items,clip,sigma,B", [(976, 40, 10, 2.3, 3), (4096, 16, 12, 2.8, 2)])
def test_pair_exact_at_worst_case_limbs(n, items, clip, sigma, B):
    """A = 0x8080 (limbs -128, -127) against S = +-c: the largest partial
    sums, on the short-K fold (n = 976: below 2^22) and on the general one
    (n = 4096: above 2^22)."""
    logq = 16
    k = 8 * items
    A_o = np.full((n, n), 0x8080, dtype=np.uint16)
    S = np.full((k, n), clip, dtype=np.int8)
    S[1::2] = -clip
    ctx = _pair_ctx(lwe.Params(n=n, logq=logq, B=B, clip=clip, sigma=sigma), items)
    out = torch.empty((k, n), dtype=torch.int16, device="cuda")
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, logq, A=dev(A_o.view(np.int16)), ctx=ctx)
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, None, logq))
    assert ctx.device_error() == 0


@pytest.mark.parametrize("name,count", [("P640", 21), ("P976", 48), ("P1344", 19)])
def test_pair_kem_matches_oracle(name, count):
    p, po = params(name)
    pk_o, sk_o, A_o, ms = oracle_keys(cfg_key(PRESETS[name]), 21)
    ctx = _pair_ctx(p, count)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
    ctx.keygen(dev(ms[None, :]), pk, sk, A_out=A)
    cs = coins(count, seed=41)
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps(pk, dev(cs), ct, K, A=A)
    K2 = torch.empty_like(K)
    ctx.decaps(sk, ct, K2, A=A)
    bad = ct.clone()
    bad[::2, 5] ^= 4
    Kb = torch.empty_like(K)
    ctx.decaps(sk, bad, Kb, A=A)
    ct_h, K_h, K2_h, Kb_h, bad_h = host(ct), host(K), host(K2), host(Kb), host(bad)
    for i in range(count):
        ct_o, K_o = O.encaps(po, pk_o, bytes(cs[i]), A=A_o)
        assert np.array_equal(ct_h[i], ct_o), i
        assert np.array_equal(K_h[i], K_o), i
    assert np.array_equal(K2_h, K_h)
    for i in (0, 1, 2, count - 1):
        assert np.array_equal(Kb_h[i], O.decaps(po, sk_o, bad_h[i], A=A_o)), i
    assert ctx.device_error() == 0


@pytest.mark.parametrize("kchunk", [64, 512])
def test_pair_ksplit_matches_oracle(kchunk):
    cfg = PRESETS["P976"]
    p, po = lwe.Params(**cfg), O.Params(**cfg)
    n, count = p.n, 35
    ctx = _pair_ctx(p, count)
    ctx.set_option(lwe.OPT_GEMM_KCHUNK, kchunk)
    r = np.random.default_rng(kchunk + 1)
    seed = r.integers(0, 256, 16, dtype=np.uint8)
    A_o = O.expand_A(bytes(seed), n, 16)
    S = r.integers(-10, 11, size=(8 * count, n), dtype=np.int8)
    E = r.integers(-10, 11, size=(8 * count, n), dtype=np.int8)
    out = torch.empty((8 * count, n), dtype=torch.int16, device="cuda")
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, 16, A=dev(A_o.view(np.int16)), E=dev(E), ctx=ctx)
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, E, 16))
    assert ctx.device_error() == 0


def test_pair_batched_4096_equals_single_cta_and_oracle():
    """The benchmarked workload on CTA pairs equals the single-CTA kernel's
    result and the oracle's, item for item (all 4096 ciphertexts and both
    key sets)."""
    name, count = "P976", 4096
    p, po = params(name)
    pk_o, sk_o, A_o, ms = oracle_keys(cfg_key(PRESETS[name]), 21)
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(lwe.PATH_TENSOR)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
    ctx.keygen(dev(ms[None, :]), pk, sk, A_out=A)
    cs = coins(count, seed=4097)
    res = {}
    for pair in (1, 0):
        ctx.set_option(lwe.OPT_GEMM_PAIR, pair)
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, dev(cs), ct, K, A=A)
        K2 = torch.empty_like(K)
        ctx.decaps(sk, ct, K2, A=A)
        res[pair] = (host(ct), host(K), host(K2))
    assert np.array_equal(res[1][0], res[0][0])
    assert np.array_equal(res[1][1], res[0][1])
    assert np.array_equal(res[1][2], res[1][1])
    ct_o, K_o = O.encaps_batch(po, pk_o, cs, A=A_o, nthreads=O.max_threads())
    bad = np.nonzero((res[1][0] != ct_o).any(axis=1))[0]
    assert bad.size == 0, "ciphertexts differ from the oracle at %s" % bad[:8]
    assert np.array_equal(res[1][1], K_o)
    K2_o = O.decaps_batch(po, sk_o, res[1][0], A=A_o, nthreads=O.max_threads())
    assert np.array_equal(res[1][2], K2_o)
    assert ctx.device_error() == 0


def test_serial_option_gives_the_same_results():
    """LWE_OPT_SERIAL (side-stream work on the caller's stream) changes the
    schedule only."""
    name, count = "P976", 40
    p, _ = params(name)
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(lwe.PATH_TENSOR)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    ctx.keygen(dev(master_seeds(1, seed=3)), pk, sk)
    cs = dev(coins(count, seed=33))
    out = []
    for serial in (0, 1):
        ctx.set_option(lwe.OPT_SERIAL, serial)
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, cs, ct, K)
        K2 = torch.empty_like(K)
        ctx.decaps(sk, ct, K2)
        out.append((host(ct), host(K), host(K2)))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], out[0][2])


@pytest.mark.parametrize("pair", [1, 0])
@pytest.mark.parametrize("group", [0, 1, 3, 8, 64])
def test_tile_group_order_matches_oracle(pair, group):
    """LWE_OPT_GEMM_GROUP changes only the order in which the persistent
    CTAs visit the output tiles: 800 rows (4 CTA-pair row blocks, the last
    with rows for one CTA only; 7 single-CTA blocks) x 976 columns (a ragged
    last column tile), groups that divide the row blocks, that leave a
    ragged last group, and that exceed them."""
    n, items = 976, 100
    k = 8 * items
    r = np.random.default_rng(group + 101 * pair)
    seed = r.integers(0, 256, 16, dtype=np.uint8)
    A_o = O.expand_A(bytes(seed), n, 16)
    S = r.integers(-10, 11, size=(k, n), dtype=np.int8)
    E = r.integers(-10, 11, size=(k, n), dtype=np.int8)
    ctx = lwe.Ctx(lwe.Params(**PRESETS["P976"]), max_batch=items)
    ctx.set_path(lwe.PATH_TENSOR)
    ctx.set_option(lwe.OPT_GEMM_PAIR, pair)
    ctx.set_option(lwe.OPT_GEMM_GROUP, group)
    out = torch.empty((k, n), dtype=torch.int16, device="cuda")
    lwe.matmul_modq(lwe.SIDE_SA, dev(S), out, n, 16, A=dev(A_o.view(np.int16)), E=dev(E), ctx=ctx)
    assert np.array_equal(as_u16(out), O.mul_SA(S, A_o, E, 16))
    assert ctx.device_error() == 0


def test_tile_group_option_range():
    ctx = lwe.Ctx(lwe.Params(**PRESETS["P640"]), max_batch=8)
    for bad in (-1, 65):
        with pytest.raises(RuntimeError):
            ctx.set_option(lwe.OPT_GEMM_GROUP, bad)
    ctx.set_option(lwe.OPT_GEMM_GROUP, 0)
