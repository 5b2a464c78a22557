"""lwe_encaps_noalloc: Encaps for callers that may not allocate device memory
(their host application owns all device allocations through its own pool, or
their request path cannot pay for an allocation).  It borrows the library's
built-in scratch area instead of a context workspace, so it must give exactly
what lwe_encaps gives.  Called here through the C ABI, twice in a row (the
area keeps the previous call's contents), against the regular entry point.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2606_01211_gb300 import lwe
from paper_2606_01211_gb300.inputs import PRESETS, coins, master_seeds

pytestmark = pytest.mark.gpu


def _noalloc(p, pk, A, cs, count, ct, K):
    cp = p.c()
    return lwe.lib().lwe_encaps_noalloc(
        C.byref(cp), pk.data_ptr(), None if A is None else A.data_ptr(), cs.data_ptr(), count,
        ct.data_ptr(), K.data_ptr(), torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("name,count", [("P640", 7), ("P976", 16)])
def test_encaps_noalloc_equals_encaps_on_two_calls(name, count):
    torch.cuda.set_device(0)
    p = lwe.Params(**PRESETS[name])
    ctx = lwe.Ctx(p, max_batch=count)
    ctx.set_path(lwe.PATH_SKINNY)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
    ctx.keygen(torch.from_numpy(master_seeds(1, seed=3)).cuda(), pk, sk, A_out=A)
    for call, useA in enumerate([A, None]):
        cs = torch.from_numpy(coins(count, seed=50 + call)).cuda()
        ct_ref = ctx.empty_ct(count)
        K_ref = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, cs, ct_ref, K_ref, A=useA)
        ct = torch.full_like(ct_ref, 0xA5)
        K = torch.full_like(K_ref, 0x5A)
        assert _noalloc(p, pk, useA, cs, count, ct, K) == lwe.LWE_OK
        torch.cuda.synchronize()
        assert torch.equal(ct, ct_ref), "ciphertexts differ on call %d" % call
        assert torch.equal(K, K_ref), "keys differ on call %d" % call
        # and they decapsulate with the regular entry point
        K2 = torch.empty_like(K)
        ctx.decaps(sk, ct, K2, A=useA)
        assert torch.equal(K2, K)


def _scratch_bytes(n, count):
    """The documented size of the scratch a call needs: its parts (seeds,
    mu, K', flags, H(pk), round keys, S', E', E'') each rounded up to 256
    bytes."""
    up = lambda b: (b + 255) // 256 * 256
    parts = [32 * count, 32 * count, 32 * count, 4 * count, 32, 176 * count,
             8 * n * count, 8 * n * count, 64 * count]
    return sum(up(b) for b in parts)


def test_encaps_noalloc_equals_tensor_path_up_to_the_largest_count():
    """A default (AUTO) context takes the tensor-core GEMM from 64 items on;
    the no-alloc call (CUDA cores) must still give the same bytes, up to the
    largest count that fits the area, and refuse one item more."""
    torch.cuda.set_device(0)
    p = lwe.Params(**PRESETS["P640"])
    cap = lwe.LWE_NOALLOC_SCRATCH_BYTES
    top = max(c for c in range(1, 200) if _scratch_bytes(p.n, c) <= cap)
    assert top >= 64
    ctx = lwe.Ctx(p, max_batch=top + 1)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda")
    ctx.keygen(torch.from_numpy(master_seeds(1, seed=8)).cuda(), pk, sk, A_out=A)
    for count in (64, 96, top):
        cs = torch.from_numpy(coins(count, seed=700 + count)).cuda()
        ct_ref = ctx.empty_ct(count)
        K_ref = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        ctx.encaps(pk, cs, ct_ref, K_ref, A=A)
        ct = torch.full_like(ct_ref, 0x3C)
        K = torch.full_like(K_ref, 0xC3)
        assert _noalloc(p, pk, A, cs, count, ct, K) == lwe.LWE_OK
        torch.cuda.synchronize()
        assert torch.equal(ct, ct_ref), "ciphertexts differ at %d items" % count
        assert torch.equal(K, K_ref), "keys differ at %d items" % count
    count = top + 1
    cs = torch.zeros((count, 32), dtype=torch.uint8, device="cuda")
    ct = torch.zeros((count, p.ct_bytes), dtype=torch.uint8, device="cuda")
    K = torch.zeros((count, 32), dtype=torch.uint8, device="cuda")
    assert _noalloc(p, pk, A, cs, count, ct, K) == lwe.LWE_ECAPACITY
    ctx.close()


def test_encaps_noalloc_allocates_no_device_memory():
    """After a first call (which does the one-time set-up), a further call
    changes neither the device's free memory nor torch's allocation count."""
    torch.cuda.set_device(0)
    p = lwe.Params(**PRESETS["P976"])
    count = 8
    ctx = lwe.Ctx(p, max_batch=1)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    ctx.keygen(torch.from_numpy(master_seeds(1, seed=9)).cuda(), pk, sk)
    cs = torch.from_numpy(coins(count, seed=9)).cuda()
    ct = ctx.empty_ct(count)
    K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
    assert _noalloc(p, pk, None, cs, count, ct, K) == lwe.LWE_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    assert _noalloc(p, pk, None, cs, count, ct, K) == lwe.LWE_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    ctx.close()


def test_encaps_noalloc_rejects_what_does_not_fit():
    torch.cuda.set_device(0)
    p = lwe.Params(**PRESETS["P4096"])
    pk = torch.zeros(p.pk_bytes, dtype=torch.uint8, device="cuda")
    count = 64  # about 4.3 MB of scratch, more than the 1 MiB area
    cs = torch.zeros((count, 32), dtype=torch.uint8, device="cuda")
    ct = torch.zeros((count, p.ct_bytes), dtype=torch.uint8, device="cuda")
    K = torch.zeros((count, 32), dtype=torch.uint8, device="cuda")
    assert _noalloc(p, pk, None, cs, count, ct, K) == lwe.LWE_ECAPACITY
    bad = lwe.Params(n=24, logq=16, B=2, clip=10, sigma=2.3)
    assert _noalloc(bad, pk, None, cs, 1, ct, K) == lwe.LWE_EINVAL
    torch.cuda.synchronize()
    assert int(K.sum()) == 0  # nothing was launched
