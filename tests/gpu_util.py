"""Helpers shared by the GPU tests: seeded inputs on the device, byte views,
and the oracle's key material computed once per parameter set."""
import functools

import numpy as np
import torch

from oracle import oracle as O
from paper_2606_01211_gb300 import lwe
from paper_2606_01211_gb300.inputs import PRESETS, coins, master_seeds


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def as_u16(t: torch.Tensor) -> np.ndarray:
    return host(t).view(np.uint16)


def params(name=None, **cfg):
    if name is not None:
        cfg = dict(PRESETS[name], **cfg)
    return lwe.Params(**cfg), O.Params(**cfg)


@functools.lru_cache(maxsize=None)
def oracle_keys(cfg_items, seed):
    """(pk, sk, A) of the oracle for a parameter set (as a tuple of items)."""
    po = O.Params(**dict(cfg_items))
    ms = master_seeds(1, seed=seed)[0]
    pk, sk, A = O.keygen(po, bytes(ms), want_A=True)
    return pk, sk, A, ms


def cfg_key(cfg: dict):
    return tuple(sorted(cfg.items()))


__all__ = ["dev", "host", "as_u16", "params", "oracle_keys", "cfg_key", "coins", "master_seeds",
           "PRESETS", "O", "lwe"]
