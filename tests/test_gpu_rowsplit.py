"""GPU parity of the row-split products (lwe_matmul_modq_rows, rowsplit.py)
against the oracle: every rank's block computed by the library's kernels on
this one GPU (A stored as the rank's row block, or regenerated from seedA),
combined by the gather / reduction rule, and compared bit for bit with the
oracle's full A S + E and S A + E; and the same through a one-rank NCCL
group.  The kernels of the ranks do not wait on one another, so running the
ranks one after another on one GPU is the same computation."""
import os
import socket

import numpy as np
import pytest
import torch

from gpu_util import O, as_u16, dev, lwe
from paper_2606_01211_gb300 import rowsplit

pytestmark = pytest.mark.gpu


def _case(n, k, seed):
    r = np.random.default_rng(seed)
    seedA = r.integers(0, 256, 16, dtype=np.uint8)
    A = O.expand_A(bytes(seedA), n, 16)
    St = r.integers(-12, 13, size=(8, n), dtype=np.int8)
    E = r.integers(-12, 13, size=(n, 8), dtype=np.int8)
    S = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    Ep = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    return seedA, A, St, E, S, Ep


@pytest.mark.parametrize("n,k,world", [(1024, 8, 2), (4096, 24, 3), (4096, 8, 5), (2048, 16, 1)])
@pytest.mark.parametrize("stored", [True, False])
def test_rank_blocks_combine_to_the_oracle_products(n, k, world, stored):
    torch.cuda.set_device(0)
    seedA, A_o, St, E, S, Ep = _case(n, k, n * 7 + k + world)
    A = dev(A_o.view(np.int16))
    sd, St_d, E_d, S_d = dev(seedA), dev(St), dev(E), dev(S)
    as_parts, sa_parts = [], []
    for rank in range(world):
        r0, r1 = rowsplit.row_block(n, world, rank)
        A_rows = A[r0:r1].contiguous() if stored else None
        as_parts.append(rowsplit.as_rows(St_d, n, 16, r0, r1, A_rows=A_rows,
                                         seedA=None if stored else sd,
                                         E_rows=E_d[r0:r1].contiguous()))
        sa_parts.append(rowsplit.sa_partial(S_d, n, 16, r0, r1, A_rows=A_rows,
                                            seedA=None if stored else sd))
    B = as_u16(rowsplit.gather_rows(as_parts))
    Bp = as_u16(rowsplit.reduce_partials(sa_parts, 16, dev(Ep)))
    assert np.array_equal(B, O.mul_AS(A_o, St, E, 16))
    assert np.array_equal(Bp, O.mul_SA(S, A_o, Ep, 16))


def test_row_blocks_reject_misaligned_ranges():
    torch.cuda.set_device(0)
    n = 256
    S = torch.zeros((8, n), dtype=torch.int8, device="cuda")
    out = torch.zeros((8, n), dtype=torch.int16, device="cuda")
    seed = torch.zeros(16, dtype=torch.uint8, device="cuda")
    for r0, r1 in ((8, 64), (0, 40), (64, 64), (0, 272)):
        with pytest.raises(lwe.LweError):
            lwe.matmul_modq_rows(lwe.SIDE_SA, S, out, n, 16, r0, r1, seedA=seed)


def test_one_rank_nccl_group_gives_the_oracle_products():
    import torch.distributed as dist
    torch.cuda.set_device(0)
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        n, k = 1024, 16
        seedA, A_o, St, E, S, Ep = _case(n, k, 99)
        g = rowsplit.RowGroup()
        B = rowsplit.keygen_B(g, dev(St), n, 16, seedA=dev(seedA), E=dev(E))
        Bp = rowsplit.encrypt_Bp(g, dev(S), n, 16, A_rows=dev(A_o.view(np.int16)), E=dev(Ep))
        assert np.array_equal(as_u16(B), O.mul_AS(A_o, St, E, 16))
        assert np.array_equal(as_u16(Bp), O.mul_SA(S, A_o, Ep, 16))
    finally:
        dist.destroy_process_group()
