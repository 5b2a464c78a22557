"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method: it only draws reproducible
random bytes (master seeds for KeyGen, coins for Encaps) and lists the
parameter sets of the workloads.  Both the CUDA path and the CPU oracle take
their inputs from here; nothing here depends on either of them.

The workloads are synthetic, as in the paper's own experiments (random keys,
Sec. 3.6 and Sec. 4): a master seed per key pair and 32 bytes of coins per
encapsulation, drawn uniformly.
"""
from __future__ import annotations

import numpy as np

# Parameter sets of the workloads (n, log2 q, message bits per coefficient B,
# clip bound c, Gaussian sigma); nbar = mbar = 8 throughout.
PRESETS = {
    "P640": dict(n=640, logq=15, B=2, clip=12, sigma=2.8),
    "P976": dict(n=976, logq=16, B=3, clip=10, sigma=2.3),
    "P1344": dict(n=1344, logq=16, B=4, clip=6, sigma=1.4),
    "P4096": dict(n=4096, logq=16, B=2, clip=12, sigma=2.8),
    "P16384": dict(n=16384, logq=16, B=1, clip=12, sigma=2.8),
    "P32768": dict(n=32768, logq=16, B=1, clip=12, sigma=2.8),
}
PRESET_IDS = {"P640": 0, "P976": 1, "P1344": 2, "P4096": 3, "P16384": 4, "P32768": 5}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_bytes(count: int, width: int, seed: int) -> np.ndarray:
    """count x width uniformly random bytes."""
    return rng(seed).integers(0, 256, size=(count, width), dtype=np.uint8)


def master_seeds(count: int, seed: int = 1) -> np.ndarray:
    """32-byte KeyGen master seeds, one per key pair."""
    return random_bytes(count, 32, 0x5EED0000 + seed)


def coins(count: int, seed: int = 1) -> np.ndarray:
    """32 bytes of Encaps randomness per encapsulation."""
    return random_bytes(count, 32, 0xC0150000 + seed)
