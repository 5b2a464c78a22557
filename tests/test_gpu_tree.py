"""The batched tree hash (H(c) in Encaps and Decaps, and the Encaps key)
under each of its launch schedules, against the oracle over whole batches:
the balanced schedule (k_tree_bal: leaves that fill 13 warps per SM, handed
between SM sub-partitions, roots absorbed in two stages) at P976 with 26
and 27 ciphertexts per SM (3801 and 4104 items, the last CTA ragged) and at
P1344 (2800 items), and the one-leaf-per-thread schedule (k_tree) just
outside that range (3800 items at P976, and P640)."""
import numpy as np
import pytest
import torch

from gpu_util import O, PRESETS, cfg_key, coins, dev, host, lwe, oracle_keys, params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,count", [("P976", 3801), ("P976", 4104), ("P1344", 2800),
                                        ("P976", 3800), ("P640", 4096)])
def test_batched_hashes_match_the_oracle(name, count):
    torch.cuda.set_device(0)
    cfg = PRESETS[name]
    p, po = params(name)
    pk_o, sk_o, A_o, ms = oracle_keys(cfg_key(cfg), 23)
    ctx = lwe.Ctx(p, max_batch=count)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
    ctx.keygen(dev(ms[None, :]), pk, sk, A_out=A)
    cs = coins(count, seed=count)
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps(pk, dev(cs), ct, K, A=A)
    bad = ct.clone()
    bad[1::2, 100] ^= 4
    K2 = torch.empty_like(K)
    ctx.decaps(sk, bad, K2, A=A)
    ct_h, K_h, K2_h, bad_h = host(ct), host(K), host(K2), host(bad)
    ct_o, K_o = O.encaps_batch(po, pk_o, cs, A=A_o, nthreads=O.max_threads())
    assert np.array_equal(ct_h, ct_o)
    assert np.array_equal(K_h, K_o)
    K2_o = O.decaps_batch(po, sk_o, bad_h, A=A_o, nthreads=O.max_threads())
    assert np.array_equal(K2_h, K2_o)
    assert np.array_equal(K2_h[0::2], K_h[0::2])      # untouched ciphertexts
    assert not (K2_h[1::2] == K_h[1::2]).all(axis=1).any()  # rejected ones
    assert ctx.device_error() == 0
