"""Decaps(Encaps(pk)) = the encapsulated key over 10^4 (key, coins) pairs per
parameter set, on the batched tensor-core path: 10 key pairs x 1000
encapsulations each.  The parameter sets' message bits per coefficient were
chosen so that decryption failures are negligible (per-operation failure
below 1e-13 by the normal estimate of the decryption noise), so every one
of the 10^4 keys must match; a ciphertext with one flipped bit must be
rejected (implicit rejection gives a different key).  Sampled items are
checked against the oracle elsewhere; this is the property at scale."""
import numpy as np
import pytest
import torch

from gpu_util import PRESETS, coins, dev, host, lwe, master_seeds

pytestmark = pytest.mark.gpu

KEYS, PER_KEY = 10, 1000


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name", ["P640", "P976", "P1344", "P4096", "P16384", "P32768"])
def test_decaps_of_encaps_over_10k_pairs(name):
    p = lwe.Params(**PRESETS[name])
    ctx = lwe.Ctx(p, max_batch=PER_KEY)
    ctx.set_path(lwe.PATH_TENSOR)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
    ct = ctx.empty_ct(PER_KEY)
    K = torch.empty((PER_KEY, 32), dtype=torch.uint8, device="cuda")
    K2 = torch.empty_like(K)
    ms = master_seeds(KEYS, seed=1000 + p.n)
    matched = 0
    for k in range(KEYS):
        ctx.keygen(dev(ms[k:k + 1]), pk, sk, A_out=A)
        cs = dev(coins(PER_KEY, seed=2000 * p.n + k))
        ctx.encaps(pk, cs, ct, K, A=A)
        ctx.decaps(sk, ct, K2, A=A)
        eq = (K == K2).all(dim=1)
        matched += int(eq.sum())
        # one flipped bit in every tenth ciphertext: rejected, all others kept
        bad = ct.clone()
        bad[::10, 3 + k] ^= 1
        Kb = torch.empty_like(K)
        ctx.decaps(sk, bad, Kb, A=A)
        rej = (Kb != K).any(dim=1)
        assert bool(rej[::10].all()), (name, k)
        keep = torch.ones(PER_KEY, dtype=torch.bool, device="cuda")
        keep[::10] = False
        assert bool((~rej[keep]).all()), (name, k)
        # the same item twice gives the same key (determinism)
        assert np.array_equal(host(K[:1]), host(K2[:1]))
    assert matched == KEYS * PER_KEY, (name, matched)
    assert ctx.device_error() == 0
