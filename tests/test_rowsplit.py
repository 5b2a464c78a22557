"""The row split of one huge-n product over several ranks (rowsplit.py):
row blocks, the all-gather of A S + E and the sum-reduction of the S A
partials.  Run here as gloo ranks on the CPU (world sizes 2 and 3, the
latter with blocks of unequal size); each rank's block product stands in
for the GPU kernel (numpy on the rank's rows of the oracle's A), and the
gathered / reduced results must equal the oracle's full products bit for
bit at n = 64 and at the P4096 dimension (n = 4096)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_01211_gb300 import rowsplit


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(n, k, seed):
    from oracle import oracle as O
    r = np.random.default_rng(seed)
    seedA = bytes(r.integers(0, 256, 16, dtype=np.uint8))
    A = O.expand_A(seedA, n, 16)
    St = r.integers(-12, 13, size=(8, n), dtype=np.int8)
    E = r.integers(-12, 13, size=(n, 8), dtype=np.int8)
    S = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    Ep = r.integers(-12, 13, size=(k, n), dtype=np.int8)
    return A, St, E, S, Ep


def _worker(rank, world, port, n, k, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A, St, E, S, Ep = _case(n, k, n + k)
    g = rowsplit.RowGroup()
    r0, r1 = g.block(n)
    q = 1 << 16
    # the rank's block products (what lwe_matmul_modq_rows computes on a GPU)
    a = A[r0:r1].astype(np.int64)
    local_as = ((a @ St.T.astype(np.int64) + E[r0:r1]) % q).astype(np.uint16)
    local_sa = ((S[:, r0:r1].astype(np.int64) @ a) % q).astype(np.uint16)
    B = g.all_gather_rows(torch.from_numpy(local_as.view(np.int16)), n)
    Bp = g.all_reduce_partial(torch.from_numpy(local_sa.view(np.int16)), 16,
                              torch.from_numpy(Ep))
    out[rank] = (r0, r1, B.numpy().view(np.uint16).copy(), Bp.numpy().view(np.uint16).copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("n,k,world", [(64, 8, 2), (4096, 16, 2), (4096, 8, 3)])
def test_row_split_products_equal_the_oracle(n, k, world):
    from oracle import oracle as O
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), n, k, out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    A, St, E, S, Ep = _case(n, k, n + k)
    want_B = O.mul_AS(A, St, E, 16)
    want_Bp = O.mul_SA(S, A, Ep, 16)
    blocks = sorted((res[r][0], res[r][1]) for r in range(world))
    assert blocks[0][0] == 0 and blocks[-1][1] == n
    assert all(b[1] == c[0] for b, c in zip(blocks, blocks[1:]))   # a partition of the rows
    for r in range(world):
        assert np.array_equal(res[r][2], want_B), r
        assert np.array_equal(res[r][3], want_Bp), r


def test_row_blocks_partition_in_aligned_groups():
    for n in (16, 64, 976, 4096, 32768):
        for world in (1, 2, 3, 5, 8, 64):
            blocks = [rowsplit.row_block(n, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in blocks]
            assert all(s % 16 == 0 for s in sizes)
            assert max(sizes) - min(sizes) <= 16


def test_local_combine_equals_the_collective_rule():
    """gather_rows / reduce_partials (one process holding every block) follow
    the same rule as the collectives: concatenation, and the integer sum
    masked mod q."""
    r = np.random.default_rng(3)
    parts = [torch.from_numpy(r.integers(0, 1 << 16, size=(8, 48), dtype=np.uint16).view(np.int16))
             for _ in range(3)]
    got = rowsplit.reduce_partials(parts, 16).numpy().view(np.uint16)
    want = sum(p.numpy().view(np.uint16).astype(np.int64) for p in parts) % (1 << 16)
    assert np.array_equal(got, want)
    rows = [torch.from_numpy(r.integers(0, 1 << 16, size=(16 * i + 16, 8), dtype=np.uint16)
                             .view(np.int16)) for i in range(3)]
    assert np.array_equal(rowsplit.gather_rows(rows).numpy(),
                          np.concatenate([x.numpy() for x in rows]))
