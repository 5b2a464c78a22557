"""ctypes binding of the plain CPU oracle (oracle/lwe_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and
bench.py's CPU-baseline leg (and its ``--impl reference`` arm) may import this
module.  The product library never loads it, and it loads nothing of the
product: it shares no code with paper_2606_01211_gb300/.

Every function mirrors one of lwe_oracle.h, which cites the passage of the
paper (Alg. 1-5, Sec. 2.1-2.2, Sec. 3.3) that it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lwe_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblwe_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and (
        os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
        and os.path.getmtime(_LIB_PATH)
        >= os.path.getmtime(os.path.join(_HERE, "lwe_oracle.h"))
    ):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-lm"]
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:] + ["-o", tmp],
                       check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


class _Params(C.Structure):
    _fields_ = [("n", C.c_uint32), ("nbar", C.c_uint32), ("mbar", C.c_uint32),
                ("logq", C.c_uint32), ("B", C.c_uint32), ("clip", C.c_uint32),
                ("sigma", C.c_double)]


class _Trace(C.Structure):
    _fields_ = [("mu", C.c_uint8 * 32), ("pkh", C.c_uint8 * 32),
                ("kprime", C.c_uint8 * 32), ("seed_se", C.c_uint8 * 16),
                ("hc", C.c_uint8 * 32), ("Sp", C.c_void_p), ("Ep", C.c_void_p),
                ("Epp", C.c_void_p), ("M", C.c_void_p), ("eq", C.c_int)]


_P = C.POINTER(_Params)
_vp = C.c_void_p
_sz = C.c_size_t
_u32 = C.c_uint32


def _declare(L):
    L.orc_aes128_key_expand.argtypes = [_vp, _vp]
    L.orc_aes128_encrypt.argtypes = [_vp, _vp, _vp]
    L.orc_ctr_block.argtypes = [_vp, C.c_uint64, C.c_uint64, _vp]
    L.orc_ctr_stream.argtypes = [_vp, C.c_uint64, C.c_uint64, _sz, _vp]
    L.orc_sha3_256.argtypes = [_vp, _sz, _vp]
    L.orc_htree.argtypes = [_vp, _sz, _vp]
    L.orc_cdf_table.argtypes = [C.c_double, _u32, _vp]
    L.orc_cdf_table.restype = C.c_int
    L.orc_sample.argtypes = [C.c_uint16, _vp, _u32]
    L.orc_sample.restype = C.c_int
    L.orc_noise.argtypes = [_vp, C.c_uint64, _vp, _u32, _sz, _vp]
    L.orc_expand_A.argtypes = [_vp, _u32, _u32, _vp]
    L.orc_mul_AS.argtypes = [_u32, _u32, _u32, _vp, _vp, _vp, _vp]
    L.orc_mul_SA.argtypes = [_u32, _u32, _u32, _u32, _vp, _vp, _vp, _vp]
    for f in ("orc_pk_bytes", "orc_sk_bytes", "orc_ct_bytes", "orc_mu_bytes"):
        getattr(L, f).argtypes = [_P]
        getattr(L, f).restype = _sz
    L.orc_check_params.argtypes = [_P]
    L.orc_keygen.argtypes = [_P, _vp, _vp, _vp, _vp]
    L.orc_encaps.argtypes = [_P, _vp, _vp, _vp, _vp, _vp]
    L.orc_decaps.argtypes = [_P, _vp, _vp, _vp, _vp]
    L.orc_encaps_trace.argtypes = [_P, _vp, _vp, _vp, _vp, _vp, C.POINTER(_Trace)]
    L.orc_decaps_trace.argtypes = [_P, _vp, _vp, _vp, _vp, C.POINTER(_Trace)]
    L.orc_keygen_batch.argtypes = [_P, _vp, _sz, _vp, _vp, C.c_int]
    L.orc_encaps_batch.argtypes = [_P, _vp, _vp, _vp, _sz, _vp, _vp, C.c_int]
    L.orc_decaps_batch.argtypes = [_P, _vp, _vp, _vp, _sz, _vp, C.c_int]
    L.orc_max_threads.restype = C.c_int


def _ptr(a):
    return None if a is None else a.ctypes.data


def _u8(b) -> np.ndarray:
    return np.frombuffer(bytes(b), dtype=np.uint8).copy()


@dataclass(frozen=True)
class Params:
    n: int
    logq: int
    B: int
    clip: int
    sigma: float
    nbar: int = 8
    mbar: int = 8

    def c(self):
        return _Params(self.n, self.nbar, self.mbar, self.logq, self.B,
                       self.clip, self.sigma)


# ---- primitives ---------------------------------------------------------

def aes128_encrypt(key: bytes, block: bytes) -> bytes:
    rk = np.zeros(176, np.uint8)
    lib().orc_aes128_key_expand(_ptr(_u8(key)), _ptr(rk))
    out = np.zeros(16, np.uint8)
    lib().orc_aes128_encrypt(_ptr(rk), _ptr(_u8(block)), _ptr(out))
    return out.tobytes()


def ctr_blocks(key: bytes, domain: int, first: int, count: int) -> bytes:
    rk = np.zeros(176, np.uint8)
    lib().orc_aes128_key_expand(_ptr(_u8(key)), _ptr(rk))
    out = np.zeros(16, np.uint8)
    res = bytearray()
    for b in range(first, first + count):
        lib().orc_ctr_block(_ptr(rk), domain, b, _ptr(out))
        res += out.tobytes()
    return bytes(res)


def ctr_stream(key: bytes, domain: int, first: int, count: int) -> np.ndarray:
    """`count` keystream blocks as one uint8 array (16 count bytes)."""
    out = np.zeros(16 * max(count, 1), np.uint8)
    if count:
        lib().orc_ctr_stream(_ptr(_u8(key)), domain, first, count, _ptr(out))
    return out[:16 * count]


def sha3_256(msg: bytes) -> bytes:
    m = _u8(msg) if len(msg) else np.zeros(1, np.uint8)
    out = np.zeros(32, np.uint8)
    lib().orc_sha3_256(_ptr(m), len(msg), _ptr(out))
    return out.tobytes()


def htree(msg: bytes) -> bytes:
    m = _u8(msg) if len(msg) else np.zeros(1, np.uint8)
    out = np.zeros(32, np.uint8)
    lib().orc_htree(_ptr(m), len(msg), _ptr(out))
    return out.tobytes()


TREE_CHUNK = 1024


def cdf_table(sigma: float, clip: int) -> np.ndarray | None:
    T = np.zeros(16, np.uint16)
    rc = lib().orc_cdf_table(sigma, clip, _ptr(T))
    return None if rc != 0 else T[:clip].copy()


def sample(w: int, T: np.ndarray, clip: int) -> int:
    TT = np.zeros(16, np.uint16)
    TT[:clip] = T[:clip]
    return int(lib().orc_sample(w, _ptr(TT), clip))


def noise(key: bytes, domain: int, T: np.ndarray, clip: int, count: int) -> np.ndarray:
    TT = np.zeros(16, np.uint16)
    TT[:clip] = T[:clip]
    out = np.zeros(max(count, 1), np.int8)
    lib().orc_noise(_ptr(_u8(key)), domain, _ptr(TT), clip, count, _ptr(out))
    return out[:count]


def expand_A(seedA: bytes, n: int, logq: int) -> np.ndarray:
    A = np.zeros((n, n), np.uint16)
    lib().orc_expand_A(_ptr(_u8(seedA)), n, logq, _ptr(A))
    return A


def mul_AS(A: np.ndarray, St: np.ndarray, E: np.ndarray | None, logq: int) -> np.ndarray:
    n = A.shape[0]
    k = St.shape[0]
    A = np.ascontiguousarray(A, np.uint16)
    St = np.ascontiguousarray(St, np.int8)
    E = None if E is None else np.ascontiguousarray(E, np.int8)
    out = np.zeros((n, k), np.uint16)
    lib().orc_mul_AS(n, k, logq, _ptr(A), _ptr(St), _ptr(E), _ptr(out))
    return out


def mul_SA(S: np.ndarray, X: np.ndarray, E: np.ndarray | None, logq: int) -> np.ndarray:
    m, n = S.shape
    ncol = X.shape[1]
    S = np.ascontiguousarray(S, np.int8)
    X = np.ascontiguousarray(X, np.uint16)
    E = None if E is None else np.ascontiguousarray(E, np.int8)
    out = np.zeros((m, ncol), np.uint16)
    lib().orc_mul_SA(m, n, ncol, logq, _ptr(S), _ptr(X), _ptr(E), _ptr(out))
    return out


# ---- KEM ----------------------------------------------------------------

def sizes(p: Params):
    cp = p.c()
    L = lib()
    return (L.orc_pk_bytes(C.byref(cp)), L.orc_sk_bytes(C.byref(cp)),
            L.orc_ct_bytes(C.byref(cp)), L.orc_mu_bytes(C.byref(cp)))


def check_params(p: Params) -> bool:
    cp = p.c()
    return lib().orc_check_params(C.byref(cp)) == 0


def keygen(p: Params, ms: bytes, want_A: bool = False):
    cp = p.c()
    pkb, skb, _, _ = sizes(p)
    pk = np.zeros(pkb, np.uint8)
    sk = np.zeros(skb, np.uint8)
    A = np.zeros((p.n, p.n), np.uint16) if want_A else None
    rc = lib().orc_keygen(C.byref(cp), _ptr(_u8(ms)), _ptr(pk), _ptr(sk), _ptr(A))
    if rc != 0:
        raise ValueError("invalid parameters")
    return (pk, sk, A) if want_A else (pk, sk)


def encaps(p: Params, pk: np.ndarray, coins: bytes, A: np.ndarray | None = None,
           trace: bool = False):
    cp = p.c()
    _, _, ctb, _ = sizes(p)
    ct = np.zeros(ctb, np.uint8)
    K = np.zeros(32, np.uint8)
    pk = np.ascontiguousarray(pk, np.uint8)
    if not trace:
        rc = lib().orc_encaps(C.byref(cp), _ptr(pk), _ptr(A), _ptr(_u8(coins)),
                              _ptr(ct), _ptr(K))
        if rc != 0:
            raise ValueError("invalid parameters")
        return ct, K
    Sp = np.zeros((p.mbar, p.n), np.int8)
    Ep = np.zeros((p.mbar, p.n), np.int8)
    Epp = np.zeros((p.mbar, p.nbar), np.int8)
    tr = _Trace()
    tr.Sp, tr.Ep, tr.Epp, tr.M = Sp.ctypes.data, Ep.ctypes.data, Epp.ctypes.data, None
    rc = lib().orc_encaps_trace(C.byref(cp), _ptr(pk), _ptr(A), _ptr(_u8(coins)),
                                _ptr(ct), _ptr(K), C.byref(tr))
    if rc != 0:
        raise ValueError("invalid parameters")
    mub = sizes(p)[3]
    info = dict(mu=bytes(tr.mu)[:mub], pkh=bytes(tr.pkh), kprime=bytes(tr.kprime),
                seed_se=bytes(tr.seed_se), hc=bytes(tr.hc), Sp=Sp, Ep=Ep, Epp=Epp)
    return ct, K, info


def decaps(p: Params, sk: np.ndarray, ct: np.ndarray, A: np.ndarray | None = None,
           trace: bool = False):
    cp = p.c()
    K = np.zeros(32, np.uint8)
    sk = np.ascontiguousarray(sk, np.uint8)
    ct = np.ascontiguousarray(ct, np.uint8)
    if not trace:
        rc = lib().orc_decaps(C.byref(cp), _ptr(sk), _ptr(A), _ptr(ct), _ptr(K))
        if rc != 0:
            raise ValueError("invalid parameters")
        return K
    M = np.zeros((p.mbar, p.nbar), np.uint16)
    tr = _Trace()
    tr.Sp = tr.Ep = tr.Epp = None
    tr.M = M.ctypes.data
    rc = lib().orc_decaps_trace(C.byref(cp), _ptr(sk), _ptr(A), _ptr(ct), _ptr(K),
                                C.byref(tr))
    if rc != 0:
        raise ValueError("invalid parameters")
    mub = sizes(p)[3]
    info = dict(mu=bytes(tr.mu)[:mub], pkh=bytes(tr.pkh), kprime=bytes(tr.kprime),
                seed_se=bytes(tr.seed_se), hc=bytes(tr.hc), M=M, eq=bool(tr.eq))
    return K, info


def keygen_batch(p: Params, ms: np.ndarray, nthreads: int = 1):
    cp = p.c()
    count = ms.shape[0]
    pkb, skb, _, _ = sizes(p)
    pk = np.zeros((count, pkb), np.uint8)
    sk = np.zeros((count, skb), np.uint8)
    ms = np.ascontiguousarray(ms, np.uint8)
    lib().orc_keygen_batch(C.byref(cp), _ptr(ms), count, _ptr(pk), _ptr(sk), nthreads)
    return pk, sk


def encaps_batch(p: Params, pk: np.ndarray, coins: np.ndarray,
                 A: np.ndarray | None = None, nthreads: int = 1):
    cp = p.c()
    count = coins.shape[0]
    _, _, ctb, _ = sizes(p)
    ct = np.zeros((count, ctb), np.uint8)
    K = np.zeros((count, 32), np.uint8)
    coins = np.ascontiguousarray(coins, np.uint8)
    pk = np.ascontiguousarray(pk, np.uint8)
    lib().orc_encaps_batch(C.byref(cp), _ptr(pk), _ptr(A), _ptr(coins), count,
                           _ptr(ct), _ptr(K), nthreads)
    return ct, K


def decaps_batch(p: Params, sk: np.ndarray, ct: np.ndarray,
                 A: np.ndarray | None = None, nthreads: int = 1):
    cp = p.c()
    count = ct.shape[0]
    K = np.zeros((count, 32), np.uint8)
    sk = np.ascontiguousarray(sk, np.uint8)
    ct = np.ascontiguousarray(ct, np.uint8)
    lib().orc_decaps_batch(C.byref(cp), _ptr(sk), _ptr(A), _ptr(ct), count,
                           _ptr(K), nthreads)
    return K


def max_threads() -> int:
    return int(lib().orc_max_threads())
