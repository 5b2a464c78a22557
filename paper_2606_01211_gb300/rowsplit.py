"""One huge-n product split by rows of A over several GPUs.

The paper runs each KEM operation on one GPU and names multi-GPU execution
as future work (Sec. 5); at n = 32768 its products are bound by the traffic
(or the regeneration) of the 2 GiB matrix A (Sec. 4.3).  Splitting A by
blocks of rows divides that work without moving A at all, because every GPU
holds -- or regenerates from seedA -- only its own rows:

  KeyGen (Alg. 1):   B = A S + E.  Row block r of B needs only row block r
                     of A: each GPU computes its rows, then ONE all-gather
                     of the n x 8 result (16 n bytes in all).
  Encrypt (Alg. 2):  B' = S' A + E'.  Every output needs every row of A:
                     each GPU forms the partial sum over its rows
                     (lwe_matmul_modq_rows, already reduced mod q), then ONE
                     sum-reduction of the 8 x n partials as int32 (NCCL has
                     no 16-bit integer sum; partials below 2^16 from up to
                     2^15 GPUs cannot overflow), E' added and the sum masked
                     mod q = 2^logq.

The row blocks are multiples of 16 rows (the kernels' alignment).  Nothing
here computes a step of the product: the per-GPU work is the library's CUDA
kernels, and this module only partitions rows and runs the collectives
(torch.distributed: NCCL between GPUs, gloo for tests on CPU ranks).
"""
from __future__ import annotations

import torch

from . import lwe

ALIGN = 16


def row_block(n: int, world: int, rank: int, align: int = ALIGN) -> tuple[int, int]:
    """Rows [row0, row1) of rank `rank` of `world`: contiguous blocks of
    whole `align`-row groups, as equal as the groups allow (ranks beyond the
    number of groups get an empty block)."""
    if n % align:
        raise ValueError("n must be a multiple of %d" % align)
    groups = n // align
    g0 = groups * rank // world
    g1 = groups * (rank + 1) // world
    return g0 * align, g1 * align


def gather_rows(parts: list[torch.Tensor]) -> torch.Tensor:
    """B from the row blocks of all ranks, in rank order."""
    return torch.cat([p.reshape(-1, 8) for p in parts], dim=0)


def reduce_partials(parts: list[torch.Tensor], logq: int,
                    E: torch.Tensor | None = None) -> torch.Tensor:
    """S A + E from the ranks' partials (each k x n, mod q): their integer
    sum plus E (or none), masked mod q (as int16 storage of uint16
    values)."""
    acc = torch.zeros(parts[0].shape, dtype=torch.int32, device=parts[0].device)
    for p in parts:
        acc += p.to(torch.int32) & 0xFFFF
    if E is not None:
        acc += E.to(torch.int32)
    return (acc & ((1 << logq) - 1)).to(torch.int16)


class RowGroup:
    """The ranks of a torch.distributed process group sharing one product."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def block(self, n: int) -> tuple[int, int]:
        return row_block(n, self.world, self.rank)

    def all_gather_rows(self, local: torch.Tensor, n: int) -> torch.Tensor:
        """The full n x 8 B from each rank's block (local: rows x 8)."""
        most = max(r1 - r0 for r0, r1 in (row_block(n, self.world, r) for r in range(self.world)))
        pad = torch.zeros((most, 8), dtype=torch.int32, device=local.device)
        pad[: local.shape[0]] = local.reshape(-1, 8).to(torch.int32) & 0xFFFF
        bufs = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(bufs, pad, group=self.group)
        parts = []
        for r, b in enumerate(bufs):
            r0, r1 = row_block(n, self.world, r)
            parts.append(b[: r1 - r0])
        return gather_rows(parts).to(torch.int16)

    def all_reduce_partial(self, local: torch.Tensor, logq: int,
                           E: torch.Tensor | None = None) -> torch.Tensor:
        """S A + E from each rank's partial sum (local: k x n, mod q); E (k x
        n int8, the same on every rank, or None) is added once, after the
        reduction."""
        acc = local.to(torch.int32) & 0xFFFF
        self.dist.all_reduce(acc, op=self.dist.ReduceOp.SUM, group=self.group)
        if E is not None:
            acc += E.to(torch.int32)
        return (acc & ((1 << logq) - 1)).to(torch.int16)


def as_rows(St: torch.Tensor, n: int, logq: int, row0: int, row1: int,
            A_rows: torch.Tensor | None = None, seedA: torch.Tensor | None = None,
            E_rows: torch.Tensor | None = None) -> torch.Tensor:
    """This GPU's rows [row0, row1) of A S + E (rows x 8, int16 storage)."""
    out = torch.zeros((row1 - row0, 8), dtype=torch.int16, device=St.device)
    if row1 > row0:
        lwe.matmul_modq_rows(lwe.SIDE_AS, St, out, n, logq, row0, row1, A_rows=A_rows,
                             seedA=seedA, E=E_rows)
    return out


def sa_partial(S: torch.Tensor, n: int, logq: int, row0: int, row1: int,
               A_rows: torch.Tensor | None = None,
               seedA: torch.Tensor | None = None) -> torch.Tensor:
    """This GPU's partial S[:, row0:row1] A[row0:row1, :] mod q (k x n)."""
    out = torch.zeros((S.shape[0], n), dtype=torch.int16, device=S.device)
    if row1 > row0:
        lwe.matmul_modq_rows(lwe.SIDE_SA, S, out, n, logq, row0, row1, A_rows=A_rows,
                             seedA=seedA)
    return out


def keygen_B(g: RowGroup, St: torch.Tensor, n: int, logq: int,
             A_rows: torch.Tensor | None = None, seedA: torch.Tensor | None = None,
             E: torch.Tensor | None = None) -> torch.Tensor:
    """B = A S + E (n x 8) over the group: own rows, then one all-gather.
    E is the full n x 8 error (each rank uses its rows); A_rows is this
    rank's block of A or None (regenerated from seedA)."""
    r0, r1 = g.block(n)
    E_rows = E[r0:r1].contiguous() if E is not None else None
    return g.all_gather_rows(as_rows(St, n, logq, r0, r1, A_rows, seedA, E_rows), n)


def encrypt_Bp(g: RowGroup, S: torch.Tensor, n: int, logq: int,
               A_rows: torch.Tensor | None = None, seedA: torch.Tensor | None = None,
               E: torch.Tensor | None = None) -> torch.Tensor:
    """B' = S' A + E' (k x n) over the group: partial over own rows, then
    one sum-reduction."""
    r0, r1 = g.block(n)
    return g.all_reduce_partial(sa_partial(S, n, logq, r0, r1, A_rows, seedA), logq, E)
