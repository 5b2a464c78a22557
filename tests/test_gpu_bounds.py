"""The bounds-checked debug build (liblwe_check.so, LWE_CHECK_BOUNDS): every
kernel tests the index arithmetic of its memory accesses against the sizes
it was given and skips and counts any access that would leave its buffer.
Here a child process loads that build and runs the hot path's kernels on
the benchmarked shape and on ragged ones; no access may have been skipped,
and the outputs must equal the product build's byte for byte."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def workload():
    """Outputs of a fixed set of calls: the headline batch on the tensor
    path (balanced tree hash, CTA-pair GEMM), a ragged CUDA-core batch with
    regenerated A, a P640 batch (dense tree schedule), a P4096 batch of
    1000 (the two-launch tree of long messages, the GEMM's grouped tile
    order), the K-split GEMM, row blocks, and the paper profile."""
    from paper_2606_01211_gb300 import lwe, rowsplit
    from paper_2606_01211_gb300.inputs import PRESETS, coins, master_seeds
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = {}
    for name, count, path, stored in (("P976", 4096, lwe.PATH_TENSOR, True),
                                      ("P640", 21, lwe.PATH_SKINNY, False),
                                      ("P1344", 19, lwe.PATH_TENSOR, False),
                                      ("P640", 4096, lwe.PATH_TENSOR, True),
                                      ("P4096", 1000, lwe.PATH_TENSOR, False)):
        p = lwe.Params(**PRESETS[name])
        ctx = lwe.Ctx(p, max_batch=count)
        ctx.set_path(path)
        pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
        A = torch.empty((p.n, p.n), dtype=torch.int16, device="cuda") if stored else None
        ctx.keygen(dev(master_seeds(1, seed=5)), pk, sk, A_out=A)
        ct = ctx.empty_ct(count)
        K = torch.empty((count, 32), dtype=torch.uint8, device="cuda")
        K2 = torch.empty_like(K)
        ctx.encaps(pk, dev(coins(count, seed=6)), ct, K, A=A)
        ctx.decaps(sk, ct, K2, A=A)
        out["%s_%d" % (name, count)] = np.concatenate(
            [pk.cpu().numpy().ravel(), sk.cpu().numpy().ravel(), ct.cpu().numpy().ravel(),
             K.cpu().numpy().ravel(), K2.cpu().numpy().ravel()])
        ctx.close()
    r = np.random.default_rng(1)
    n = 2048
    seed = dev(r.integers(0, 256, 16, dtype=np.uint8))
    S = dev(r.integers(-12, 13, size=(64 * 8, n), dtype=np.int8))
    o = torch.empty((64 * 8, n), dtype=torch.int16, device="cuda")
    p2 = lwe.Params(n=n, logq=16, B=1, clip=12, sigma=2.8)
    c2 = lwe.Ctx(p2, max_batch=64)
    c2.set_path(lwe.PATH_TENSOR)
    c2.set_option(lwe.OPT_GEMM_KCHUNK, 512)
    lwe.matmul_modq(lwe.SIDE_SA, S, o, n, 16, seedA=seed, ctx=c2)
    out["ksplit"] = o.cpu().numpy().ravel()
    parts = [rowsplit.sa_partial(S[:8].contiguous(), n, 16, *rowsplit.row_block(n, 3, k),
                                 seedA=seed) for k in range(3)]
    out["rows"] = rowsplit.reduce_partials(parts, 16).cpu().numpy().ravel()
    c2.close()
    pp = lwe.PpParams("PP512")
    pc = lwe.PpCtx(pp)
    ppk, psk, pA, pct = pc.empty_pk(), pc.empty_sk(), pc.empty_A(), pc.empty_ct()
    pK = torch.empty(32, dtype=torch.uint8, device="cuda")
    pc.keygen(dev(np.arange(32, dtype=np.uint8)), ppk, psk, pA)
    pc.encaps(ppk, pA, dev(np.arange(32, 64, dtype=np.uint8)), pct, pK)
    out["pp"] = np.concatenate([pct.cpu().numpy(), pK.cpu().numpy()])
    pc.close()
    torch.cuda.synchronize()
    return out


@pytest.mark.gpu
def test_checked_build_skips_no_access_and_gives_the_same_bytes():
    from paper_2606_01211_gb300 import build_lib
    build_lib.build(check_bounds=True)
    torch.cuda.set_device(0)
    want = workload()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "checked.npz")
        env = dict(os.environ, LWE_CHECK_BOUNDS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), path], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stdout + r.stderr
        got = dict(np.load(path))
    viol = got.pop("violations")
    assert int(viol[0]) == 0, "skipped accesses: %d, first at site %d" % (viol[0], viol[1])
    assert set(got) == set(want)
    for k in want:
        assert np.array_equal(got[k], want[k]), k


if __name__ == "__main__":
    from paper_2606_01211_gb300 import lwe
    assert lwe.bounds_violations() == (0, 0), "not the checked build, or stale counts"
    torch.cuda.set_device(0)
    res = workload()
    res["violations"] = np.array(lwe.bounds_violations(), dtype=np.int64)
    np.savez(sys.argv[1], **res)
