"""Batched KEM against one public key, replayed from CUDA graphs, and the
tile autotuner.

BatchedKem holds one key pair, its expanded A and static input/output
buffers for a fixed batch; its step (Encaps of the batch followed by the
Decaps of the produced ciphertexts) is captured once into a CUDA graph and
replayed, so a step costs one graph launch on the host instead of ~30
kernel launches.  The key is bound to the context (lwe_ctx_bind_key), so its
H(pk) and the limb split of [A | B] are made once, not in every step.
Batching many encapsulations against one key is what turns S' A into one
tensor-core contraction (the paper batches the 256
per-bit encryptions of one Encaps into one launch, Sec. 3.2).

autotune() times the candidate GEMM kernels (CTA pairs on 256 x 128 tiles,
or one CTA on 128 x 64 / 128 x 128 tiles) and the items-per-call threshold
above which the tensor path beats the CUDA-core path, for a given (n,
batch), and caches the choice in a JSON file.
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import lwe
from .inputs import PRESETS, coins as make_coins, master_seeds

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")


class BatchedKem:
    def __init__(self, name: str = "P976", count: int = 4096, seed: int = 1, device=None,
                 path: int = lwe.PATH_TENSOR, gemm_bn: int | None = None,
                 gemm_pair: int | None = None, bind: bool = True):
        self.dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.params = p = lwe.Params(**PRESETS[name])
        self.count = count
        self.ctx = lwe.Ctx(p, max_batch=count, device=self.dev.index)
        self.ctx.set_path(path)
        if gemm_bn:
            self.ctx.set_option(lwe.OPT_GEMM_BN, gemm_bn)
        if gemm_pair is not None:
            self.ctx.set_option(lwe.OPT_GEMM_PAIR, gemm_pair)
        self.pk, self.sk = self.ctx.empty_pk(1), self.ctx.empty_sk(1)
        self.A = torch.empty((p.n, p.n), dtype=torch.int16, device=self.dev)
        self.ctx.keygen(torch.from_numpy(master_seeds(1, seed=seed)).to(self.dev), self.pk, self.sk,
                        A_out=self.A)
        if bind:  # H(pk) and the limbs of [A | B], made once for the key
            self.ctx.bind_key(self.pk, self.sk, self.A)
        self.coins = torch.from_numpy(make_coins(count, seed=seed)).to(self.dev)
        self.ct = self.ctx.empty_ct(count)
        self.K = torch.empty((count, 32), dtype=torch.uint8, device=self.dev)
        self.K2 = torch.empty_like(self.K)
        self.graph = None

    def step(self):
        """Encaps of the batch, then Decaps of its ciphertexts, on the
        current stream."""
        self.ctx.encaps(self.pk, self.coins, self.ct, self.K, A=self.A)
        self.ctx.decaps(self.sk, self.ct, self.K2, A=self.A)

    def capture(self, timing: bool = False):
        """Capture one step.  With timing, CUDA events around every kernel
        are captured too; call timed_replay_done() after each completed
        replay to add the kernels' durations to the context statistics."""
        s = torch.cuda.Stream(device=self.dev)
        s.wait_stream(torch.cuda.current_stream(self.dev))
        if timing:  # creates the event pairs outside the capture
            self.ctx.set_option(lwe.OPT_TIMING, 1)
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream(self.dev).wait_stream(s)
        torch.cuda.synchronize(self.dev)
        if timing:
            self.ctx.set_option(lwe.OPT_TIMING, 0)
            self.ctx.reset_stats()
        g = torch.cuda.CUDAGraph()
        launches0 = self.ctx.launches()
        if timing:
            self.ctx.set_option(lwe.OPT_TIMING, 1)
        with torch.cuda.graph(g):
            self.step()
        if timing:
            self.ctx.set_option(lwe.OPT_TIMING, 0)
            self.ctx.timing_mark()
        torch.cuda.synchronize(self.dev)
        self.launches_per_step = self.ctx.launches() - launches0
        self.graph = g
        return g

    def timed_replay_done(self):
        self.ctx.timing_replay()

    def replay(self, coins: torch.Tensor | None = None):
        """One step from the captured graph; new coins are copied into the
        static input buffer first."""
        if coins is not None:
            self.coins.copy_(coins, non_blocking=True)
        self.graph.replay()

    def close(self):
        self.graph = None
        self.ctx.close()


def _time(fn, reps: int = 5) -> float:
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def autotune(name: str = "P976", count: int = 4096, cache: str | None = CACHE,
             refresh: bool = False) -> dict:
    """Pick the GEMM tile width and the tensor-path threshold for (n, batch).

    Returns {"gemm_pair": 0|1, "gemm_bn": 64|128, "tensor_min": items,
    "ms": {...}} and stores it under the key "<name>/<count>" in the cache
    file."""
    key = "%s/%d" % (name, count)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table and not refresh and "gemm_pair" in table[key]:
            return table[key]
    kem = BatchedKem(name, count, path=lwe.PATH_TENSOR)
    ms = {}
    cands = {"tensor_pair": (1, 128), "tensor_bn128": (0, 128), "tensor_bn64": (0, 64)}
    for label, (pair, bn) in cands.items():
        kem.ctx.set_option(lwe.OPT_GEMM_PAIR, pair)
        kem.ctx.set_option(lwe.OPT_GEMM_BN, bn)
        ms[label] = _time(kem.step)
    best = min(cands, key=lambda k: ms[k])
    best_pair, best_bn = cands[best]
    kem.ctx.set_option(lwe.OPT_GEMM_PAIR, best_pair)
    kem.ctx.set_option(lwe.OPT_GEMM_BN, best_bn)
    # crossover: smallest batch at which the tensor path is faster per item
    tensor_min = count + 1
    for b in (16, 32, 64, 128, 256, 512, 1024, 2048, 4096):
        if b > count:
            break
        t = {}
        for path in (lwe.PATH_SKINNY, lwe.PATH_TENSOR):
            kem.ctx.set_path(path)
            t[path] = _time(lambda: (kem.ctx.encaps(kem.pk, kem.coins[:b], kem.ct[:b], kem.K[:b],
                                                    A=kem.A)), reps=3)
        ms["encaps%d_skinny" % b], ms["encaps%d_tensor" % b] = t[lwe.PATH_SKINNY], t[lwe.PATH_TENSOR]
        if t[lwe.PATH_TENSOR] < t[lwe.PATH_SKINNY]:
            tensor_min = b
            break
    kem.close()
    res = {"gemm_pair": best_pair, "gemm_bn": best_bn, "tensor_min": tensor_min, "ms": ms}
    if cache:
        table[key] = res
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return res
