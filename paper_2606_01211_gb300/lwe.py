"""Python binding of liblwe.so (include/lwe.h): argument marshalling only.

Every function takes torch CUDA tensors (uint8 / int8 / int16 storage),
checks their sizes, and passes their device pointers and the current CUDA
stream to the C ABI.  All arithmetic of the KEM runs in the library's CUDA
kernels; nothing here computes any step of it, and there is no CPU fallback:
if liblwe.so is missing or fails to load, import raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

from .build_lib import LIB, LIB_CHECK

# LWE_CHECK_BOUNDS=1 selects the bounds-checked debug build of the library
# (build it first with build_lib.build(check_bounds=True))
_LIB_PATH = LIB_CHECK if os.environ.get("LWE_CHECK_BOUNDS") == "1" else LIB

# status codes (include/lwe.h)
LWE_OK = 0
LWE_EINVAL = -1
LWE_ENOMEM = -2
LWE_ECUDA = -3
LWE_ETIMEOUT = -4
LWE_EUNSUPPORTED = -5
LWE_ECAPACITY = -6
LWE_NOALLOC_SCRATCH_BYTES = 1024 * 1024  # the built-in scratch of lwe_encaps_noalloc

PATH_AUTO, PATH_SKINNY, PATH_TENSOR = 0, 1, 2
(OPT_PATH, OPT_TENSOR_MIN, OPT_TIMING, OPT_GEMM_BN, OPT_GEMM_KCHUNK, OPT_GEMM_PAIR,
 OPT_SERIAL, OPT_WARP_HASH_MAX, OPT_PDL, OPT_GEMM_GROUP) = 0, 1, 2, 3, 4, 5, 6, 7, 8, 9
SIDE_AS, SIDE_SA = 0, 1
PRESET_IDS = {"P640": 0, "P976": 1, "P1344": 2, "P4096": 3, "P16384": 4, "P32768": 5}


class LweError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = "%s failed: %s (%d)" % (what, _lib.lwe_strerror(code).decode(), code)
        if code == LWE_ECUDA:
            msg += ": " + _lib.lwe_last_cuda_error().decode()
        super().__init__(msg)
        self.code = code


class _Params(C.Structure):
    _fields_ = [("n", C.c_uint32), ("nbar", C.c_uint32), ("mbar", C.c_uint32),
                ("logq", C.c_uint32), ("B", C.c_uint32), ("clip", C.c_uint32),
                ("sigma", C.c_double)]


class _PpParams(C.Structure):
    _fields_ = [("n", C.c_uint32), ("q", C.c_uint32), ("k", C.c_uint32), ("clip", C.c_uint32),
                ("sigma", C.c_double)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError("%s is not built (run __graft_entry__.build() or "
                          "python -m paper_2606_01211_gb300.build_lib)" % os.path.basename(_LIB_PATH))
    lib = C.CDLL(_LIB_PATH)
    vp, u32, i32, sz = C.c_void_p, C.c_uint32, C.c_int, C.c_size_t
    P = C.POINTER(_Params)
    PP = C.POINTER(_PpParams)
    sig = {
        "lwe_params_preset": (i32, [i32, P]),
        "lwe_params_check": (i32, [P]),
        "lwe_cdf_table": (i32, [P, vp]),
        "lwe_pk_bytes": (sz, [P]),
        "lwe_sk_bytes": (sz, [P]),
        "lwe_ct_bytes": (sz, [P]),
        "lwe_ctx_create": (i32, [P, u32, i32, C.POINTER(vp)]),
        "lwe_ctx_destroy": (i32, [vp]),
        "lwe_ctx_set_option": (i32, [vp, i32, C.c_int64]),
        "lwe_keygen": (i32, [vp, vp, u32, vp, vp, vp, vp]),
        "lwe_encaps": (i32, [vp, vp, vp, vp, u32, vp, vp, vp]),
        "lwe_decaps": (i32, [vp, vp, vp, vp, u32, vp, vp]),
        "lwe_encaps_multi": (i32, [vp, vp, vp, vp, vp, u32, vp, vp, vp]),
        "lwe_decaps_multi": (i32, [vp, vp, vp, vp, u32, vp, vp]),
        "lwe_ctx_bind_key": (i32, [vp, vp, vp, vp, vp]),
        "lwe_expand_A": (i32, [vp, u32, u32, vp, vp]),
        "lwe_matmul_modq": (i32, [vp, i32, vp, vp, vp, u32, u32, u32, vp, vp, vp]),
        "lwe_matmul_modq_rows": (i32, [i32, vp, vp, vp, u32, u32, u32, u32, u32, vp, vp, vp]),
        "lwe_encaps_noalloc": (i32, [P, vp, vp, vp, u32, vp, vp, vp]),
        "lwe_selftest_bounded_wait": (i32, [vp, u32, vp]),
        "lwe_probe": (i32, [i32, u32, u32, vp, vp]),
        "lwe_noise_table": (i32, [P, vp, vp]),
        "lwe_bounds_violations": (i32, [C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
        "lwe_strerror": (C.c_char_p, [i32]),
        "lwe_last_cuda_error": (C.c_char_p, []),
        "lwe_ctx_device_error": (i32, [vp]),
        "lwe_ctx_launches": (C.c_uint64, [vp]),
        "lwe_ctx_kernel_stats": (i32, [vp, i32, C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
        "lwe_ctx_reset_stats": (i32, [vp]),
        "lwe_ctx_timing_mark": (i32, [vp]),
        "lwe_ctx_timing_replay": (i32, [vp]),
        "lwe_kernel_name": (C.c_char_p, [i32]),
        "lwe_num_kernels": (i32, []),
        "lwe_pp_params_preset": (i32, [i32, PP]),
        "lwe_pp_params_check": (i32, [PP]),
        "lwe_pp_pk_bytes": (sz, [PP]),
        "lwe_pp_sk_bytes": (sz, [PP]),
        "lwe_pp_ct_bytes": (sz, [PP]),
        "lwe_pp_ctx_create": (i32, [PP, i32, C.POINTER(vp)]),
        "lwe_pp_ctx_destroy": (i32, [vp]),
        "lwe_pp_ctx_set_option": (i32, [vp, i32, C.c_int64]),
        "lwe_pp_expand_A": (i32, [PP, vp, vp, vp]),
        "lwe_pp_keygen": (i32, [vp, vp, vp, vp, vp, vp]),
        "lwe_pp_encaps": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "lwe_pp_decaps": (i32, [vp, vp, vp, vp, vp, vp]),
        "lwe_pp_ctx_bind_key": (i32, [vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc: int, what: str):
    if rc != LWE_OK:
        raise LweError(rc, what)


@dataclass(frozen=True)
class Params:
    n: int
    logq: int
    B: int
    clip: int
    sigma: float
    nbar: int = 8
    mbar: int = 8

    def c(self) -> _Params:
        return _Params(self.n, self.nbar, self.mbar, self.logq, self.B, self.clip, self.sigma)

    @staticmethod
    def preset(name: str) -> "Params":
        p = _Params()
        _check(_lib.lwe_params_preset(PRESET_IDS[name], C.byref(p)), "lwe_params_preset")
        return Params(n=p.n, logq=p.logq, B=p.B, clip=p.clip, sigma=p.sigma)

    def valid(self) -> bool:
        cp = self.c()
        return _lib.lwe_params_check(C.byref(cp)) == LWE_OK

    @property
    def pk_bytes(self) -> int:
        cp = self.c()
        return int(_lib.lwe_pk_bytes(C.byref(cp)))

    @property
    def sk_bytes(self) -> int:
        cp = self.c()
        return int(_lib.lwe_sk_bytes(C.byref(cp)))

    @property
    def ct_bytes(self) -> int:
        cp = self.c()
        return int(_lib.lwe_ct_bytes(C.byref(cp)))

    def cdf_table(self):
        import numpy as np
        T = np.zeros(16, np.uint16)
        cp = self.c()
        _check(_lib.lwe_cdf_table(C.byref(cp), T.ctypes.data), "lwe_cdf_table")
        return T[: self.clip].copy()


def _ptr(t: torch.Tensor | None, dtype=None, nbytes: int | None = None, what: str = "") -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must have dtype %s, got %s" % (what, dtype, t.dtype))
    if nbytes is not None and t.numel() * t.element_size() < nbytes:
        raise ValueError("%s holds %d bytes, needs %d" % (what, t.numel() * t.element_size(), nbytes))
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Ctx:
    """An lwe_ctx: parameters, device workspaces for max_batch items."""

    def __init__(self, params: Params, max_batch: int = 1, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.params = params
        self.max_batch = max_batch
        self.device = device
        h = C.c_void_p()
        cp = params.c()
        _check(_lib.lwe_ctx_create(C.byref(cp), max_batch, device, C.byref(h)), "lwe_ctx_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.lwe_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        _check(_lib.lwe_ctx_set_option(self._h, option, int(value)), "lwe_ctx_set_option")

    def set_path(self, path: int):
        self.set_option(OPT_PATH, path)

    def device_error(self) -> int:
        return int(_lib.lwe_ctx_device_error(self._h))

    def launches(self) -> int:
        return int(_lib.lwe_ctx_launches(self._h))

    def kernel_stats(self) -> dict:
        out = {}
        for k in range(_lib.lwe_num_kernels()):
            n = C.c_uint64()
            ms = C.c_double()
            _check(_lib.lwe_ctx_kernel_stats(self._h, k, C.byref(n), C.byref(ms)), "kernel_stats")
            if n.value:
                out[_lib.lwe_kernel_name(k).decode()] = (int(n.value), float(ms.value))
        return out

    def reset_stats(self):
        _check(_lib.lwe_ctx_reset_stats(self._h), "lwe_ctx_reset_stats")

    def timing_mark(self):
        _check(_lib.lwe_ctx_timing_mark(self._h), "lwe_ctx_timing_mark")

    def timing_replay(self):
        _check(_lib.lwe_ctx_timing_replay(self._h), "lwe_ctx_timing_replay")

    # ---- buffers -------------------------------------------------------
    def empty_pk(self, count: int = 1) -> torch.Tensor:
        return torch.empty((count, self.params.pk_bytes), dtype=torch.uint8, device="cuda")

    def empty_sk(self, count: int = 1) -> torch.Tensor:
        return torch.empty((count, self.params.sk_bytes), dtype=torch.uint8, device="cuda")

    def empty_ct(self, count: int = 1) -> torch.Tensor:
        return torch.empty((count, self.params.ct_bytes), dtype=torch.uint8, device="cuda")

    def bind_key(self, pk: torch.Tensor | None, sk: torch.Tensor | None = None,
                 A: torch.Tensor | None = None, stream=None):
        """Make H(pk) and the tensor path's limbs of [A | B] once for calls
        with these (pk, A) / (sk, A) buffers; bind_key(None) unbinds."""
        p = self.params
        rc = _lib.lwe_ctx_bind_key(
            self._h, _ptr(pk, torch.uint8, p.pk_bytes, "pk"), _ptr(sk, torch.uint8, p.sk_bytes, "sk"),
            _ptr(A, torch.int16, p.n * p.n * 2, "A"), _stream(stream))
        _check(rc, "lwe_ctx_bind_key")

    # ---- KEM -----------------------------------------------------------
    def keygen(self, seeds: torch.Tensor, pk: torch.Tensor, sk: torch.Tensor,
               A_out: torch.Tensor | None = None, stream=None):
        count = seeds.shape[0] if seeds.dim() > 1 else seeds.numel() // 32
        p = self.params
        rc = _lib.lwe_keygen(
            self._h, _ptr(seeds, torch.uint8, 32 * count, "seeds"), count,
            _ptr(pk, torch.uint8, count * p.pk_bytes, "pk"),
            _ptr(sk, torch.uint8, count * p.sk_bytes, "sk"),
            _ptr(A_out, torch.int16, count * p.n * p.n * 2, "A_out"), _stream(stream))
        _check(rc, "lwe_keygen")

    def encaps(self, pk: torch.Tensor, coins: torch.Tensor, ct: torch.Tensor, K: torch.Tensor,
               A: torch.Tensor | None = None, stream=None):
        count = coins.shape[0] if coins.dim() > 1 else coins.numel() // 32
        p = self.params
        rc = _lib.lwe_encaps(
            self._h, _ptr(pk, torch.uint8, p.pk_bytes, "pk"),
            _ptr(A, torch.int16, p.n * p.n * 2, "A"),
            _ptr(coins, torch.uint8, 32 * count, "coins"), count,
            _ptr(ct, torch.uint8, count * p.ct_bytes, "ct"),
            _ptr(K, torch.uint8, 32 * count, "K"), _stream(stream))
        _check(rc, "lwe_encaps")

    def encaps_multi(self, pk_ptrs: torch.Tensor, coins: torch.Tensor, ct: torch.Tensor,
                     K: torch.Tensor, pkh_ptrs: torch.Tensor | None = None,
                     A_ptrs: torch.Tensor | None = None, count: int | None = None, stream=None):
        """Item e against its own key: pk_ptrs / pkh_ptrs / A_ptrs are device
        int64 tensors of device pointers (the data_ptr() of each key)."""
        p = self.params
        if count is None:
            count = coins.shape[0]
        rc = _lib.lwe_encaps_multi(
            self._h, _ptr_array(pk_ptrs, count, "pk_ptrs"), _ptr_array(pkh_ptrs, count, "pkh_ptrs"),
            _ptr_array(A_ptrs, count, "A_ptrs"), _ptr(coins, torch.uint8, 32 * count, "coins"),
            count, _ptr(ct, torch.uint8, count * p.ct_bytes, "ct"),
            _ptr(K, torch.uint8, 32 * count, "K"), _stream(stream))
        _check(rc, "lwe_encaps_multi")

    def decaps_multi(self, sk_ptrs: torch.Tensor, ct: torch.Tensor, K: torch.Tensor,
                     A_ptrs: torch.Tensor | None = None, count: int | None = None, stream=None):
        p = self.params
        if count is None:
            count = ct.shape[0]
        rc = _lib.lwe_decaps_multi(
            self._h, _ptr_array(sk_ptrs, count, "sk_ptrs"), _ptr_array(A_ptrs, count, "A_ptrs"),
            _ptr(ct, torch.uint8, count * p.ct_bytes, "ct"), count,
            _ptr(K, torch.uint8, 32 * count, "K"), _stream(stream))
        _check(rc, "lwe_decaps_multi")

    def decaps(self, sk: torch.Tensor, ct: torch.Tensor, K: torch.Tensor,
               A: torch.Tensor | None = None, stream=None, count: int | None = None):
        p = self.params
        if count is None:
            count = ct.shape[0] if ct.dim() > 1 else ct.numel() // p.ct_bytes
        rc = _lib.lwe_decaps(
            self._h, _ptr(sk, torch.uint8, p.sk_bytes, "sk"),
            _ptr(A, torch.int16, p.n * p.n * 2, "A"),
            _ptr(ct, torch.uint8, count * p.ct_bytes, "ct"), count,
            _ptr(K, torch.uint8, 32 * count, "K"), _stream(stream))
        _check(rc, "lwe_decaps")


def _ptr_array(ptrs: torch.Tensor | None, count: int, what: str) -> int | None:
    if ptrs is None:
        return None
    if ptrs.dtype != torch.int64 or not ptrs.is_cuda or ptrs.numel() < count:
        raise ValueError("%s must be a CUDA int64 tensor of at least %d pointers" % (what, count))
    return ptrs.data_ptr()


def expand_A(seedA: torch.Tensor, n: int, logq: int, A_out: torch.Tensor, stream=None):
    """A (n x n, int16 storage of uint16 values) from a 16-byte device seed."""
    rc = _lib.lwe_expand_A(_ptr(seedA, torch.uint8, 16, "seedA"), n, logq,
                           _ptr(A_out, torch.int16, n * n * 2, "A_out"), _stream(stream))
    _check(rc, "lwe_expand_A")


def matmul_modq(side: int, S: torch.Tensor, out: torch.Tensor, n: int, logq: int,
                A: torch.Tensor | None = None, seedA: torch.Tensor | None = None,
                E: torch.Tensor | None = None, ctx: Ctx | None = None, stream=None):
    """side AS: out[n][8] = A S + E (S given as S^T, 8 x n);
    side SA: out[k][n] = S A + E (S k x n)."""
    k = S.shape[0]
    rc = _lib.lwe_matmul_modq(
        ctx.handle if ctx is not None else None, side,
        _ptr(A, torch.int16, n * n * 2, "A"), _ptr(seedA, torch.uint8, 16, "seedA"),
        _ptr(S, torch.int8, k * n, "S"), n, k, logq, _ptr(E, torch.int8, k * n, "E"),
        _ptr(out, torch.int16, k * n * 2, "out"), _stream(stream))
    _check(rc, "lwe_matmul_modq")


def noise_table(params: Params, out: torch.Tensor, stream=None):
    """The noise kernel's word table: out[w] = the sample of 16-bit word w
    (out: 65536 int8 on the device)."""
    cp = params.c()
    _check(_lib.lwe_noise_table(C.byref(cp), _ptr(out, torch.int8, 65536, "out"), _stream(stream)),
           "lwe_noise_table")


def matmul_modq_rows(side: int, S: torch.Tensor, out: torch.Tensor, n: int, logq: int,
                     row0: int, row1: int, A_rows: torch.Tensor | None = None,
                     seedA: torch.Tensor | None = None, E: torch.Tensor | None = None,
                     stream=None):
    """The products over rows [row0, row1) of A only (lwe_matmul_modq_rows):
    side AS: out[row1 - row0][8] = those rows of A S + E (E: those rows);
    side SA: out[k][n] = (S[:, row0:row1] A[row0:row1] + E) mod q.
    A_rows is the row block (row1 - row0 x n) or None (regenerated)."""
    k = S.shape[0]
    nrows = row1 - row0
    if side == SIDE_AS:
        e_bytes, o_bytes = nrows * 8, nrows * 8 * 2
    else:
        e_bytes, o_bytes = k * n, k * n * 2
    rc = _lib.lwe_matmul_modq_rows(
        side, _ptr(A_rows, torch.int16, max(nrows, 0) * n * 2, "A_rows"),
        _ptr(seedA, torch.uint8, 16, "seedA"), _ptr(S, torch.int8, k * n, "S"), n, k, logq,
        row0, row1, _ptr(E, torch.int8, e_bytes, "E"), _ptr(out, torch.int16, o_bytes, "out"),
        _stream(stream))
    _check(rc, "lwe_matmul_modq_rows")


def bounds_violations():
    """(skipped accesses, first site id) of the bounds-checked build since
    the last call; None for the product build (no checks)."""
    n, site = C.c_uint64(), C.c_uint32()
    rc = _lib.lwe_bounds_violations(C.byref(n), C.byref(site))
    if rc == LWE_EUNSUPPORTED:
        return None
    _check(rc, "lwe_bounds_violations")
    return int(n.value), int(site.value)


def kernel_names():
    return [_lib.lwe_kernel_name(i).decode() for i in range(_lib.lwe_num_kernels())]


PROBE_KECCAK, PROBE_AES, PROBE_KECCAK_WARP, PROBE_AES_RUN = 0, 1, 2, 3


def probe(kind: int, ctas: int, iters: int, sink: torch.Tensor, stream=None):
    """Measurement probe (lwe_probe): Keccak-f in registers or AES blocks
    with the shared-memory tables, no memory traffic; sink is an int32
    device tensor of at least ctas * 512 words."""
    _check(_lib.lwe_probe(kind, ctas, iters, _ptr(sink, torch.int32, ctas * 512 * 4, "sink"),
                          _stream(stream)), "lwe_probe")


# ---- the paper's own parameter profile (lwe_pp.h) ---------------------------
PP_OPT_TENSOR, PP_OPT_PDL = 0, 1
PP_PRESET_IDS = {"PP512": 0, "PP1024": 1, "PP2048": 2, "PP4096": 3, "PP8192": 4, "PP16384": 5,
                 "PP32768": 6}


class PpParams:
    """Tab. 1 parameters: n, odd q, Gaussian sigma (clip), e2 bound k."""

    def __init__(self, name: str | None = None, n: int = 0, q: int = 0, sigma: float = 0.0,
                 k: int = 0, clip: int = 0):
        self._c = _PpParams()
        if name is not None:
            _check(_lib.lwe_pp_params_preset(PP_PRESET_IDS[name], C.byref(self._c)),
                   "lwe_pp_params_preset")
        else:
            self._c.n, self._c.q, self._c.sigma, self._c.k, self._c.clip = n, q, sigma, k, clip
            _check(_lib.lwe_pp_params_check(C.byref(self._c)), "lwe_pp_params_check")
        self.n, self.q, self.sigma = self._c.n, self._c.q, self._c.sigma
        self.k, self.clip = self._c.k, self._c.clip
        self.pk_bytes = int(_lib.lwe_pp_pk_bytes(C.byref(self._c)))
        self.sk_bytes = int(_lib.lwe_pp_sk_bytes(C.byref(self._c)))
        self.ct_bytes = int(_lib.lwe_pp_ct_bytes(C.byref(self._c)))


def pp_expand_A(p: PpParams, seedA: torch.Tensor, A: torch.Tensor, stream=None):
    _check(_lib.lwe_pp_expand_A(C.byref(p._c), _ptr(seedA, torch.uint8, 16, "seedA"),
                                _ptr(A, torch.int32, 4 * p.n * p.n, "A"), _stream(stream)),
           "lwe_pp_expand_A")


class PpCtx:
    """Workspace of the paper-profile KEM; one call at a time.  A is an
    n x n int32 tensor holding the uint32 entries mod q."""

    def __init__(self, p: PpParams, device: int | None = None):
        self.params = p
        h = C.c_void_p()
        dev = torch.cuda.current_device() if device is None else device
        _check(_lib.lwe_pp_ctx_create(C.byref(p._c), dev, C.byref(h)), "lwe_pp_ctx_create")
        self._h = h

    def close(self):
        if self._h:
            _lib.lwe_pp_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensor(self, on: bool):
        """Encrypt's product on the tensor cores (default) or the CUDA cores."""
        _check(_lib.lwe_pp_ctx_set_option(self._h, PP_OPT_TENSOR, int(on)), "lwe_pp_ctx_set_option")

    def set_option(self, option: int, value: int):
        _check(_lib.lwe_pp_ctx_set_option(self._h, option, int(value)), "lwe_pp_ctx_set_option")

    def bind_key(self, pk=None, A=None, stream=None):
        """Make H(pk) and A's limbs once for later calls with these buffers;
        bind_key() unbinds."""
        p = self.params
        _check(_lib.lwe_pp_ctx_bind_key(self._h, _ptr(pk, torch.uint8, p.pk_bytes, "pk"),
                                        _ptr(A, torch.int32, 4 * p.n * p.n, "A"),
                                        _stream(stream)), "lwe_pp_ctx_bind_key")

    def empty_pk(self):
        return torch.empty(self.params.pk_bytes, dtype=torch.uint8, device="cuda")

    def empty_sk(self):
        return torch.empty(self.params.sk_bytes, dtype=torch.uint8, device="cuda")

    def empty_ct(self):
        return torch.empty(self.params.ct_bytes, dtype=torch.uint8, device="cuda")

    def empty_A(self):
        n = self.params.n
        return torch.empty((n, n), dtype=torch.int32, device="cuda")

    def keygen(self, seed32, pk, sk, A, stream=None):
        p = self.params
        _check(_lib.lwe_pp_keygen(self._h, _ptr(seed32, torch.uint8, 32, "seed"),
                                  _ptr(pk, torch.uint8, p.pk_bytes, "pk"),
                                  _ptr(sk, torch.uint8, p.sk_bytes, "sk"),
                                  _ptr(A, torch.int32, 4 * p.n * p.n, "A"), _stream(stream)),
               "lwe_pp_keygen")

    def encaps(self, pk, A, coins32, ct, K, stream=None):
        p = self.params
        _check(_lib.lwe_pp_encaps(self._h, _ptr(pk, torch.uint8, p.pk_bytes, "pk"),
                                  _ptr(A, torch.int32, 4 * p.n * p.n, "A"),
                                  _ptr(coins32, torch.uint8, 32, "coins"),
                                  _ptr(ct, torch.uint8, p.ct_bytes, "ct"),
                                  _ptr(K, torch.uint8, 32, "K"), _stream(stream)),
               "lwe_pp_encaps")

    def decaps(self, sk, A, ct, K, stream=None):
        p = self.params
        _check(_lib.lwe_pp_decaps(self._h, _ptr(sk, torch.uint8, p.sk_bytes, "sk"),
                                  _ptr(A, torch.int32, 4 * p.n * p.n, "A"),
                                  _ptr(ct, torch.uint8, p.ct_bytes, "ct"),
                                  _ptr(K, torch.uint8, 32, "K"), _stream(stream)),
               "lwe_pp_decaps")
