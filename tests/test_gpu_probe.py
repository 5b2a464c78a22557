"""Measurement probes (lwe_probe): the work they time is the real
permutation / cipher, checked on a few threads against independent
definitions -- Keccak-f[1600] written here from FIPS 202 Sec. 3.2 (pinned
by SHA3-256 against hashlib on the CPU), AES-128 from the oracle."""
import hashlib

import numpy as np
import pytest

from oracle import oracle as O

M64 = (1 << 64) - 1


def _rc_bit(t):
    """FIPS 202 Algorithm 5: the LFSR x^8 + x^6 + x^5 + x^4 + 1."""
    if t % 255 == 0:
        return 1
    r = 0x80
    for _ in range(t % 255):
        r = ((r >> 1) ^ (0x8E if r & 1 else 0)) & 0xFF
    return r >> 7


def _round_constants():
    out = []
    for ir in range(24):
        rc = 0
        for j in range(7):
            rc |= _rc_bit(j + 7 * ir) << ((1 << j) - 1)
        out.append(rc)
    return out


def _rho_offsets():
    off = [[0] * 5 for _ in range(5)]
    x, y = 1, 0
    for t in range(24):
        off[x][y] = ((t + 1) * (t + 2) // 2) % 64
        x, y = y, (2 * x + 3 * y) % 5
    return off


RC, RHO = _round_constants(), _rho_offsets()


def _rot(v, r):
    r %= 64
    return ((v << r) | (v >> (64 - r))) & M64 if r else v


def keccak_f(lanes):
    """Keccak-f[1600] on 25 lanes indexed x + 5y (FIPS 202 Sec. 3.2)."""
    A = [[lanes[x + 5 * y] for y in range(5)] for x in range(5)]
    for ir in range(24):
        C = [A[x][0] ^ A[x][1] ^ A[x][2] ^ A[x][3] ^ A[x][4] for x in range(5)]
        D = [C[(x - 1) % 5] ^ _rot(C[(x + 1) % 5], 1) for x in range(5)]
        A = [[A[x][y] ^ D[x] for y in range(5)] for x in range(5)]
        B = [[0] * 5 for _ in range(5)]
        for x in range(5):
            for y in range(5):
                B[y][(2 * x + 3 * y) % 5] = _rot(A[x][y], RHO[x][y])
        A = [[B[x][y] ^ ((~B[(x + 1) % 5][y] & M64) & B[(x + 2) % 5][y]) for y in range(5)]
             for x in range(5)]
        A[0][0] ^= RC[ir]
    return [A[i % 5][i // 5] for i in range(25)]


def _sha3_256(msg: bytes) -> bytes:
    rate = 136
    m = bytearray(msg) + b"\x06" + bytes((-len(msg) - 1) % rate)
    m[-1] |= 0x80
    s = [0] * 25
    for o in range(0, len(m), rate):
        for i in range(rate // 8):
            s[i] ^= int.from_bytes(m[o + 8 * i:o + 8 * i + 8], "little")
        s = keccak_f(s)
    return b"".join(v.to_bytes(8, "little") for v in s[:4])


def test_keccak_f_definition_matches_sha3():
    for msg in (b"", b"abc", bytes(range(200))):
        assert _sha3_256(msg) == hashlib.sha3_256(msg).digest()


def _keccak_probe_word(gid, iters):
    s = [((gid << 32) ^ ((i * 0x9E3779B9) & 0xFFFFFFFF)) & M64 for i in range(25)]
    for _ in range(iters):
        s = keccak_f(s)
    return (s[0] ^ s[7] ^ s[24]) & 0xFFFFFFFF


def _aes_probe_word(gid, iters):
    kw = [gid, (gid * 0x9E3779B9) & 0xFFFFFFFF, ~gid & 0xFFFFFFFF, gid ^ 0x5A5A5A5A]
    key = b"".join(w.to_bytes(4, "little") for w in kw)
    acc = 0
    for b in range(gid * iters, gid * iters + iters):
        blk = O.aes128_encrypt(key, (3).to_bytes(8, "big") + b.to_bytes(8, "big"))
        for i in range(4):
            acc ^= int.from_bytes(blk[4 * i:4 * i + 4], "little")
    return acc


def _aes_run_probe_word(gid, iters):
    """The windowed probe: thread gid's block i has counter index
    32 (warp iters + i) + lane, so a warp's 32 lanes cover runs of
    consecutive indices, under one key per warp, as a warp of the noise
    kernel does."""
    w = gid >> 5
    kw = [w, (w * 0x9E3779B9) & 0xFFFFFFFF, ~w & 0xFFFFFFFF, w ^ 0x5A5A5A5A]
    key = b"".join(w.to_bytes(4, "little") for w in kw)
    acc = 0
    for i in range(iters):
        b = 32 * ((gid >> 5) * iters + i) + (gid & 31)
        blk = O.aes128_encrypt(key, (3).to_bytes(8, "big") + b.to_bytes(8, "big"))
        for k in range(4):
            acc ^= int.from_bytes(blk[4 * k:4 * k + 4], "little")
    return acc


@pytest.mark.gpu
@pytest.mark.parametrize("kind,threads,iters", [(0, 256, 1), (0, 256, 3), (1, 512, 2), (1, 512, 6),
                                                (3, 512, 8), (3, 512, 16)])
def test_probe_matches_definition(kind, threads, iters):
    import torch
    from paper_2606_01211_gb300 import lwe
    torch.cuda.set_device(0)
    ctas = 2
    sink = torch.zeros(ctas * 512, dtype=torch.int32, device="cuda")
    lwe.probe(kind, ctas, iters, sink)
    torch.cuda.synchronize()
    got = sink.cpu().numpy().view(np.uint32)
    ref = {lwe.PROBE_KECCAK: _keccak_probe_word, lwe.PROBE_AES: _aes_probe_word,
           lwe.PROBE_AES_RUN: _aes_run_probe_word}[kind]
    for gid in (0, 1, 37, threads, 8 * 32 + 31, ctas * threads - 1):
        assert int(got[gid]) == ref(gid, iters), (kind, gid)


@pytest.mark.gpu
@pytest.mark.parametrize("iters", [1, 2])
def test_warp_probe_matches_definition(iters):
    """One state per warp (lane t of the state on thread t, threads 25..31
    mirroring 0..6): the same permutation as the definition."""
    import torch
    from paper_2606_01211_gb300 import lwe
    torch.cuda.set_device(0)
    ctas = 3
    sink = torch.zeros(ctas * 512, dtype=torch.int32, device="cuda")
    lwe.probe(lwe.PROBE_KECCAK_WARP, ctas, iters, sink)
    torch.cuda.synchronize()
    got = sink.cpu().numpy().view(np.uint32)
    for g in range(ctas):
        s = [((g << 32) ^ ((t * 0x9E3779B9) & 0xFFFFFFFF)) & M64 for t in range(25)]
        for _ in range(iters):
            s = keccak_f(s)
        for lane in range(32):
            v = s[lane % 25]
            assert int(got[32 * g + lane]) == (v ^ (v >> 32)) & 0xFFFFFFFF, (g, lane)


@pytest.mark.gpu
def test_probe_rejects_bad_arguments():
    import torch
    from paper_2606_01211_gb300 import lwe
    torch.cuda.set_device(0)
    sink = torch.zeros(512, dtype=torch.int32, device="cuda")
    for kind, ctas, iters in ((3, 1, 2), (0, 0, 2), (1, 1, 3)):
        with pytest.raises(Exception):
            lwe.probe(kind, ctas, iters, sink)
    with pytest.raises(ValueError):
        lwe.probe(0, 2, 1, sink)  # sink too small for two CTAs
