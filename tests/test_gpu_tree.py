"""The batched tree hash (H(c) in Encaps and Decaps, and the Encaps key)
under each of its launch schedules, against the oracle over whole batches:
- the balanced schedule (k_tree_bal: leaves that fill 13 warps per SM,
  handed between SM sub-partitions, roots absorbed in two stages) at P976
  with 26 and 27 ciphertexts per SM (3801 and 4104 items, the last CTA
  ragged) and at P1344 (2800 items);
- the dense schedule (k_tree_dense: leaves of at most 12 warps packed one
  per thread, roots on the least loaded sub-partition) at P976 with 25, 14
  and 2 ciphertexts per SM (3800: 12 leaf warps; 2048; 300: one leaf warp)
  and at P640 (4096: 9 leaf warps);
- the one-leaf-per-thread schedule (k_tree) beyond both: P1344 with 27
  ciphertexts per SM (567 leaves) and P640 with 40 per SM;
- for long messages (more than 32 chunks) k_tree while it takes one wave
  of CTAs (P4096 with 300 items, 65 chunks per ciphertext), and below, the
  two-launch schedule (every leaf on its own thread, digests in global
  memory, one warp per root) beyond that wave (P4096 with 1000 items) and
  for root chains of more than 128 chunks (P16384, 257 chunks)."""
import numpy as np
import pytest
import torch

from gpu_util import O, PRESETS, cfg_key, coins, dev, host, lwe, master_seeds, oracle_keys, params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,count", [("P976", 3801), ("P976", 4104), ("P1344", 2800),
                                        ("P976", 3800), ("P640", 4096), ("P976", 2048),
                                        ("P976", 300), ("P1344", 4096), ("P640", 6000),
                                        ("P4096", 300)])
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


def test_keygen_of_a_large_batch_hashes_every_pk():
    """KeyGen of 4096 P976 key pairs: H(pk) of all of them in one batched
    tree launch (the balanced schedule, digest mode, written into sk);
    every digest equals the oracle's tree hash of the GPU's pk, and sampled
    key pairs equal the oracle's in full."""
    torch.cuda.set_device(0)
    name, count = "P976", 4096
    p, po = params(name)
    ms = master_seeds(count, seed=77)
    ctx = lwe.Ctx(p, max_batch=count)
    pk, sk = ctx.empty_pk(count), ctx.empty_sk(count)
    ctx.keygen(dev(ms), pk, sk)
    pk_h, sk_h = host(pk), host(sk)
    off = 8 * p.n + 32
    for i in range(count):
        assert sk_h[i, off:off + 32].tobytes() == O.htree(pk_h[i].tobytes()), i
    for i in (0, 1, 2047, 4050, count - 1):   # 4050: the last, smaller CTA
        pk_o, sk_o = O.keygen(po, bytes(ms[i]))
        assert np.array_equal(pk_h[i], pk_o) and np.array_equal(sk_h[i], sk_o), i
    assert ctx.device_error() == 0


def test_multi_key_encaps_hashes_each_pk_in_one_batch():
    """lwe_encaps_multi over 4096 items with per-item public keys and no
    precomputed H(pk): the keys are hashed by pointer in one batched tree
    launch (the balanced schedule); the results equal those of the same call
    given each key's stored H(pk), and sampled items equal the oracle's."""
    torch.cuda.set_device(0)
    name, count, nk = "P976", 4096, 3
    p, po = params(name)
    ms = master_seeds(nk, seed=78)
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(lwe.PATH_SKINNY)
    pk, sk = ctx.empty_pk(nk), ctx.empty_sk(nk)
    ctx.keygen(dev(ms), pk, sk)
    keys = np.random.default_rng(79).integers(0, nk, size=count)
    pk_ptrs = torch.tensor([pk[k].data_ptr() for k in keys], dtype=torch.int64, device="cuda")
    pkh_ptrs = torch.tensor([sk[k].data_ptr() + 8 * p.n + 32 for k in keys], dtype=torch.int64,
                            device="cuda")
    cs = coins(count, seed=80)
    out = []
    for give in (None, pkh_ptrs):
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps_multi(pk_ptrs, dev(cs), ct, K, pkh_ptrs=give)
        out.append((host(ct), host(K)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    for i in (0, 3000, count - 1):
        pk_o, _ = O.keygen(po, bytes(ms[keys[i]]))
        ct_o, K_o = O.encaps(po, pk_o, bytes(cs[i]))
        assert np.array_equal(out[0][0][i], ct_o) and np.array_equal(out[0][1][i], K_o), i
    assert ctx.device_error() == 0


@pytest.mark.parametrize("name,count", [("P4096", 1000), ("P16384", 160)])
def test_long_message_tree_hashes(name, count):
    """Batches of long messages on the two-launch schedule:
    KeyGen's H(pk) of every key equals the oracle's tree hash of the GPU's
    pk; Decaps of tampered ciphertexts returns H(z || H(c)) with H(c) the
    oracle's tree hash, for every item; Decaps of the untampered ones
    returns Encaps' key, whose H(K' || H(c)) comes from the root warps."""
    torch.cuda.set_device(0)
    p, po = params(name)
    n = p.n
    ctx = lwe.Ctx(p, max_batch=count)
    ms = master_seeds(count, seed=91)
    pk, sk = ctx.empty_pk(count), ctx.empty_sk(count)
    ctx.keygen(dev(ms), pk, sk)
    pk_h, sk_h = host(pk), host(sk)
    off = 8 * n + 32
    for i in range(count):
        assert sk_h[i, off:off + 32].tobytes() == O.htree(pk_h[i].tobytes()), i
    ctx.set_path(lwe.PATH_TENSOR)
    cs = coins(count, seed=92)
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    ctx.encaps(pk[:1], dev(cs), ct, K)
    K2 = torch.empty_like(K)
    ctx.decaps(sk[:1], ct, K2)
    assert torch.equal(K, K2)
    bad = ct.clone()
    bad[:, 7] ^= 1
    Kb = torch.empty_like(K)
    ctx.decaps(sk[:1], bad, Kb)
    Kb_h, bad_h = host(Kb), host(bad)
    z = sk_h[0, 8 * n:8 * n + 32].tobytes()
    for i in range(count):
        assert Kb_h[i].tobytes() == O.sha3_256(z + O.htree(bad_h[i].tobytes())), i
    assert ctx.device_error() == 0


def test_multi_key_long_public_keys_hashed_by_pointer():
    """lwe_encaps_multi over 1000 P4096 items with per-item public keys and
    no precomputed H(pk): the keys' tree hashes (65 chunks each) go through
    the two-launch schedule by pointer; the results equal those of the same
    call given each key's stored H(pk), and a sampled item equals the
    oracle's."""
    torch.cuda.set_device(0)
    name, count, nk = "P4096", 1000, 3
    p, po = params(name)
    ms = master_seeds(nk, seed=81)
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(lwe.PATH_SKINNY)
    pk, sk = ctx.empty_pk(nk), ctx.empty_sk(nk)
    ctx.keygen(dev(ms), pk, sk)
    keys = np.random.default_rng(82).integers(0, nk, size=count)
    pk_ptrs = torch.tensor([pk[k].data_ptr() for k in keys], dtype=torch.int64, device="cuda")
    pkh_ptrs = torch.tensor([sk[k].data_ptr() + 8 * p.n + 32 for k in keys], dtype=torch.int64,
                            device="cuda")
    cs = coins(count, seed=83)
    out = []
    for give in (None, pkh_ptrs):
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps_multi(pk_ptrs, dev(cs), ct, K, pkh_ptrs=give)
        out.append((host(ct), host(K)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    i = 777
    pk_o, _ = O.keygen(po, bytes(ms[keys[i]]))
    ct_o, K_o = O.encaps(po, pk_o, bytes(cs[i]))
    assert np.array_equal(out[0][0][i], ct_o) and np.array_equal(out[0][1][i], K_o)
    assert ctx.device_error() == 0
