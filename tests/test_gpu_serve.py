"""The continuous-batching server gives every request exactly the result it
gets alone: each served Encaps equals a standalone Encaps with the same key
and coins (and decapsulates to the same key), each served Decaps returns
the key its ciphertext was made with, each served KeyGen equals a standalone
KeyGen of the same seed -- whatever batch, slot, A-cache state (stored or
regenerated A) and path the request happened to be served with.  Sampled
results are also checked against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import O, PRESETS, host, lwe
from paper_2606_01211_gb300 import serve

pytestmark = pytest.mark.gpu


NAMES = {640: "P640", 976: "P976", 1344: "P1344", 4096: "P4096"}


@pytest.fixture(scope="module")
def served():
    """The served mix over all four dimensions, with an A cache far too
    small for the keys (cache pressure: regenerated A and evictions)."""
    torch.cuda.set_device(0)
    cfg = serve.ServeConfig(presets=("P640", "P976", "P1344", "P4096"), keys_per_n=24,
                            requests=700, rate=3e4, max_batch=96, slots=3,
                            a_budget_bytes=40 << 20, seed=5)
    eng = serve.Engine(cfg)
    eng.warmup()
    stats = eng.run()
    torch.cuda.synchronize()
    return eng, stats


@pytest.fixture(scope="module")
def hot():
    """Few keys and a burst of arrivals: one key has many waiting requests,
    so single-key batches of at least 64 items take the tensor-core path."""
    torch.cuda.set_device(0)
    cfg = serve.ServeConfig(presets=("P640", "P976"), keys_per_n=3, requests=1500, rate=1e7,
                            max_batch=256, slots=2, seed=6)
    eng = serve.Engine(cfg)
    eng.warmup()
    stats = eng.run()
    torch.cuda.synchronize()
    return eng, stats


def test_serving_completes_with_batching_and_cache_pressure(served):
    eng, st = served
    assert st["requests"] == 700 and st["ops_per_s"] > 0
    assert st["mean_batch"] > 1.0          # requests were actually batched
    assert st["a_cache_misses"] > 0        # cache pressure: some A regenerated
    assert st["multi_key_batches"] > 0
    assert 0.0 < st["gpu_busy"] <= 1.0
    assert all(q.t_done >= q.t_arr for q in eng.reqs)


def test_hot_key_batches_take_the_tensor_path(hot):
    eng, st = hot
    assert st["tensor_batches"] > 0
    assert st["single_key_batches"] > 0


def _check_standalone(eng):
    ctxs = {}
    for q in eng.reqs:
        n = q.n
        p = eng.store.params[n]
        if n not in ctxs:
            c = lwe.Ctx(p, max_batch=1)
            c.set_path(lwe.PATH_SKINNY)
            ctxs[n] = c
        c = ctxs[n]
        op = serve.OPS[q.op]
        row = eng.pool[n]["row"][q.rid]
        if op == "keygen":
            pk, sk = c.empty_pk(1), c.empty_sk(1)
            c.keygen(eng.pool[n]["seeds"][row:row + 1], pk, sk)
            got_pk, got_sk = eng.result(q)
            assert torch.equal(pk[0], got_pk) and torch.equal(sk[0], got_sk), q
        elif op == "encaps":
            ct, K = c.empty_ct(1), torch.empty((1, 32), dtype=torch.uint8, device="cuda")
            c.encaps(eng.store.pk[n][q.key], eng.pool[n]["coins"][row:row + 1], ct, K)
            got_ct, got_K = eng.result(q)
            assert torch.equal(ct[0], got_ct) and torch.equal(K[0], got_K), q
            K2 = torch.empty_like(K)
            c.decaps(eng.store.sk[n][q.key], got_ct.unsqueeze(0), K2)
            assert torch.equal(K2[0], got_K), q
        else:
            got_K, want_K = eng.result(q)
            assert torch.equal(got_K, want_K), q


def test_hot_key_results_equal_their_standalone_results(hot):
    _check_standalone(hot[0])


def test_every_served_result_equals_its_standalone_result(served):
    _check_standalone(served[0])


def test_sampled_served_results_equal_the_oracle(served):
    eng, _ = served
    seen = set()
    for q in eng.reqs:
        op = serve.OPS[q.op]
        if (op, q.n) in seen or op == "decaps":
            continue
        seen.add((op, q.n))
        name = NAMES[q.n]
        po = O.Params(**PRESETS[name])
        row = eng.pool[q.n]["row"][q.rid]
        if op == "keygen":
            ms = bytes(host(eng.pool[q.n]["seeds"][row]))
            pk_o, sk_o = O.keygen(po, ms)
            got_pk, got_sk = eng.result(q)
            assert np.array_equal(host(got_pk), pk_o) and np.array_equal(host(got_sk), sk_o)
        else:
            pk = host(eng.store.pk[q.n][q.key])
            c = bytes(host(eng.pool[q.n]["coins"][row]))
            ct_o, K_o = O.encaps(po, pk, c)
            got_ct, got_K = eng.result(q)
            assert np.array_equal(host(got_ct), ct_o) and np.array_equal(host(got_K), K_o)
    assert len(seen) == 2 * len(eng.cfg.presets)


def test_plain_per_request_serving_gives_the_same_results(served):
    eng, _ = served
    cfg = serve.ServeConfig(**{**eng.cfg.__dict__, "plain": True, "requests": 120})
    plain = serve.Engine(cfg, store=eng.store)
    st = plain.run()
    assert st["mean_batch"] == 1.0
    for q in plain.reqs:
        a = plain.result(q)
        b = eng.result(eng.reqs[q.rid])
        for x, y in zip(a, b):
            assert torch.equal(x, y), q
