"""The C-ABI library loads, exports every symbol include/lwe.h declares, and
its host-only functions agree with the oracle.  No GPU is needed: nothing
here launches a kernel."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_01211_gb300 import lwe
from paper_2606_01211_gb300.inputs import PRESETS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(lwe_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_hot_path_entry_points():
    names = _declared_functions()
    for must in ["lwe_keygen", "lwe_encaps", "lwe_decaps", "lwe_expand_A", "lwe_matmul_modq",
                 "lwe_ctx_create", "lwe_ctx_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    L = C.CDLL(lwe.LIB)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("name", list(PRESETS))
def test_presets_match_the_workload_parameters(name):
    p = lwe.Params.preset(name)
    cfg = PRESETS[name]
    assert (p.n, p.logq, p.B, p.clip) == (cfg["n"], cfg["logq"], cfg["B"], cfg["clip"])
    assert abs(p.sigma - cfg["sigma"]) < 1e-12
    assert p.valid()


@pytest.mark.parametrize("name", list(PRESETS))
def test_library_noise_table_equals_oracle_table(name):
    cfg = PRESETS[name]
    p = lwe.Params(**cfg)
    assert np.array_equal(p.cdf_table(), O.cdf_table(cfg["sigma"], cfg["clip"]))


@pytest.mark.parametrize("name", list(PRESETS))
def test_object_sizes_equal_oracle_sizes(name):
    cfg = PRESETS[name]
    p = lwe.Params(**cfg)
    pkb, skb, ctb, _ = O.sizes(O.Params(**cfg))
    assert (p.pk_bytes, p.sk_bytes, p.ct_bytes) == (pkb, skb, ctb)


def test_invalid_parameters_rejected_on_the_host():
    bad = [
        lwe.Params(n=24, logq=16, B=2, clip=10, sigma=2.3),      # n % 16
        lwe.Params(n=64, logq=16, B=5, clip=10, sigma=2.3),      # B > 4
        lwe.Params(n=64, logq=3, B=3, clip=10, sigma=2.3),       # B >= logq
        lwe.Params(n=64, logq=16, B=2, clip=15, sigma=0.6),      # degenerate table
        lwe.Params(n=64, logq=16, B=2, clip=0, sigma=2.3),
        lwe.Params(n=64, logq=16, B=2, clip=10, sigma=-1.0),
    ]
    for p in bad:
        assert not p.valid()


def test_argument_errors_need_no_gpu():
    L = lwe.lib()
    assert L.lwe_expand_A(None, 64, 16, None, None) == lwe.LWE_EINVAL
    assert L.lwe_matmul_modq(None, 0, None, None, None, 64, 8, 16, None, None, None) == lwe.LWE_EINVAL
    assert L.lwe_keygen(None, None, 1, None, None, None, None) == lwe.LWE_EINVAL
    assert L.lwe_encaps(None, None, None, None, 1, None, None, None) == lwe.LWE_EINVAL
    assert L.lwe_decaps(None, None, None, None, 1, None, None) == lwe.LWE_EINVAL
    h = C.c_void_p()
    bad = lwe.Params(n=24, logq=16, B=2, clip=10, sigma=2.3).c()
    assert L.lwe_ctx_create(C.byref(bad), 1, 0, C.byref(h)) == lwe.LWE_EINVAL
    assert not h.value
    assert L.lwe_ctx_destroy(None) == lwe.LWE_OK
    assert L.lwe_strerror(lwe.LWE_ECAPACITY).decode().startswith("count exceeds")
    assert lwe.bounds_violations() is None  # the product build has no checks
    names = lwe.kernel_names()
    assert "k_gemm_tc" in names and "k_noise" in names
