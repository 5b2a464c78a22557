"""The noise kernel's sampler table against the oracle's sampler, for every
16-bit word.

k_noise turns each 16-bit keystream word into a sample through a 64 KB table
that every CTA builds in shared memory from the CDF table T (Sec. 2.2,
Tab. 1: rounded-Gaussian noise by inverse sampling).  lwe_noise_table runs
that same table build and lookup for all 65536 words, so this is an
exhaustive check of the device sampler, not a sample of it through the KEM."""
import numpy as np
import pytest
import torch

from gpu_util import O, PRESETS, lwe

pytestmark = pytest.mark.gpu

EXTRA = {
    "clip15": dict(n=64, logq=16, B=2, clip=15, sigma=4.0),
    "clip1": dict(n=64, logq=16, B=2, clip=1, sigma=0.4),
}


@pytest.mark.parametrize("name", list(PRESETS) + list(EXTRA))
def test_device_sampler_table_equals_oracle_for_every_word(name):
    torch.cuda.set_device(0)
    cfg = PRESETS.get(name) or EXTRA[name]
    p = lwe.Params(**cfg)
    assert p.valid()
    out = torch.empty(65536, dtype=torch.int8, device="cuda")
    lwe.noise_table(p, out)
    got = out.cpu().numpy()
    T = O.cdf_table(cfg["sigma"], cfg["clip"])
    want = np.array([O.sample(w, T, cfg["clip"]) for w in range(65536)], dtype=np.int8)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "words %s: device %s, oracle %s" % (bad[:4], got[bad[:4]], want[bad[:4]])
    # every magnitude 0..clip occurs, with both signs
    assert set(np.unique(want).tolist()) == set(range(-cfg["clip"], cfg["clip"] + 1))
