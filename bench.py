"""Benchmark of the batched plain-LWE KEM hot path on GB300.

Workload (one step): one P976 public key (n = 976, q = 2^16, sigma = 2.3,
c = 10, B = 3), 4096 Encaps against it (stacked S' on the tensor-core path)
followed by the 4096 matching Decaps, captured once as a CUDA graph and
replayed with each step's coins.  Inputs (keys, expanded A, the coins of
every step) are resident in HBM before the timed region; L2 is flushed
between timed steps.  value = Encaps+Decaps pairs per second over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the plain CPU oracle (oracle/) on the host cores on a
bounded sample of the same workload.  For N > 1 (torchrun) every rank runs an
independent replica (no collective on the data path) and rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_01211_gb300.inputs import PRESETS, coins, master_seeds  # noqa: E402

METRIC = "Encaps+Decaps ops/s at n=976 batched/served vs plain; p50/p99 latency; A·S GB/s"
UNIT = "Encaps+Decaps pairs/s"
PRESET = "P976"
COUNT = 4096
WORKLOAD = "batched P976 KEM: 4096 Encaps + 4096 Decaps against one public key (stored A)"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region.  Each
    sample carries nvidia-smi's timestamp, so that stop(t0, t1) keeps the
    samples taken between two host wall-clock times (the timed region)."""

    def __init__(self, index: int, period_ms: int = 200):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []

    def start(self, wait_first: bool = False):
        """wait_first: return once the first sample has arrived, so that
        sampling is live when the timed region begins (at most 5 s)."""
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
            return
        t_end = time.time() + 5.0
        while wait_first and not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    @staticmethod
    def _when(stamp: str):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(stamp, fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self, t0: float | None = None, t1: float | None = None):
        """Median SM clock, the maximum clock and the throttle reasons seen.
        With t0, t1 (time.time() around the timed region) only the samples
        inside it count; when the region is shorter than the sampling
        period, the samples just before and after it stand in and
        `in_region` says so."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(max(0.25, 2 * self.period_ms / 1e3))
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 10:
                rows.append((self._when(f[0]), f))
        picked, in_region = rows, None
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
            in_region = len(inside)
            if inside:
                picked = inside
            else:  # the nearest sample on each side of a short region
                before = [r for r in rows if r[0] is not None and r[0] < t0][-1:]
                after = [r for r in rows if r[0] is not None and r[0] > t1][:1]
                picked = before + after
        sm, smax, reasons, watts = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, f in picked:
            try:
                sm.append(float(f[2]))
                smax = float(f[3])
            except ValueError:
                continue
            try:
                watts.append(float(f[4]))
            except ValueError:
                pass
            for nm, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        self.watts = watts
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
               "reasons": sorted(reasons), "samples": len(sm)}
        if in_region is not None:
            out["in_region"] = in_region
            out["period_ms"] = self.period_ms
        return out


# ------------------------------------------------------------ reference ---
def cpu_oracle_rate(target_s: float = 12.0, max_pairs: int | None = None,
                    single_thread: bool = False):
    """The plain oracle (as it stands) on all host cores (or on one) over a
    bounded sample of the workload: Encaps + Decaps pairs per second."""
    from oracle import oracle as O
    cfg = PRESETS[PRESET]
    po = O.Params(**cfg)
    pk, sk, A = O.keygen(po, bytes(master_seeds(1, seed=1)[0]), want_A=True)
    threads = len(os.sched_getaffinity(0))
    threads = min(threads, O.max_threads()) if O.max_threads() > 1 else 1
    if single_thread:
        threads = 1
    n = max(threads, 8)
    elapsed, done = 0.0, 0
    while True:
        cs = coins(n, seed=1000 + done)
        t0 = time.perf_counter()
        ct, K = O.encaps_batch(po, pk, cs, A=A, nthreads=threads)
        K2 = O.decaps_batch(po, sk, ct, A=A, nthreads=threads)
        dt = time.perf_counter() - t0
        assert np.array_equal(K, K2)
        elapsed += dt
        done += n
        if elapsed >= target_s or (max_pairs and done >= max_pairs):
            break
        n = max(1, int(n * min(4.0, max(1.5, (target_s - elapsed) / max(dt, 1e-3)))))
        if max_pairs:
            n = min(n, max_pairs - done)
    return done / elapsed, threads, done, elapsed


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    total_pairs = 0
    threads = 1
    if args.ref_step_s is None:
        args.ref_step_s = min(8.0, 150.0 / (args.warmup + args.steps))
    for i in range(args.warmup + args.steps):
        rate, threads, pairs, el = cpu_oracle_rate(target_s=args.ref_step_s)
        if i >= args.warmup:
            steps.append((pairs, el))
            total_pairs += pairs
    tot_t = sum(e for _, e in steps)
    value = total_pairs / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic (seeded random keys and coins)",
        "config": {"workload": WORKLOAD, "n": PRESETS[PRESET]["n"], "batch": COUNT},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d Encaps+Decaps pairs per step (P976, A given), about %.0f s "
                                   "of CPU work per step" % (total_pairs // args.steps, args.ref_step_s)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def cpu_large_n(threads: int, batch: int = 1024):
    """The oracle at n = 16384 and 32768 (the sizes the paper calls
    impractical on the CPU, Sec. 4.3): one Encaps + Decaps pair per host
    thread, timed once on all threads, with A given.  pk, sk and A are
    random bytes of the right sizes: the oracle's work (S' A, S' B, the
    noise, the hashes, the re-encryption and compare) does not depend on
    their values, and expanding a 2 GiB A with its byte-wise AES would
    dominate the sample.  The batch of `batch` Encaps + Decaps is then
    extrapolated linearly from that sample (labelled)."""
    from oracle import oracle as O
    out = {}
    r = np.random.default_rng(12)
    for name in ("P16384", "P32768"):
        po = O.Params(**PRESETS[name])
        n = po.n
        pkb, skb, _, _ = O.sizes(po)
        A = r.integers(0, 1 << 16, size=(n, n), dtype=np.uint16)
        pk = r.integers(0, 256, size=pkb, dtype=np.uint8)
        sk = r.integers(0, 256, size=skb, dtype=np.uint8)
        sk[: 8 * n] = r.integers(-2, 3, size=8 * n, dtype=np.int8).view(np.uint8)
        sk[8 * n + 64:] = pk
        cs = coins(threads, seed=77)
        t0 = time.perf_counter()
        ct, _ = O.encaps_batch(po, pk, cs, A=A, nthreads=threads)
        O.decaps_batch(po, sk, ct, A=A, nthreads=threads)
        el = time.perf_counter() - t0
        rate = threads / el
        out[name] = {"pairs_per_s": rate, "sample_pairs": threads, "sample_s": el,
                     "batch_%d_s_extrapolated" % batch: batch / rate}
        del A
    out["cores"] = threads
    out["kind"] = "oracle, timed sample; batch time extrapolated linearly in the batch size"
    return out


def per_request_rate(kem, lwe, torch, stream, pairs: int = 2048):
    """The plain per-request GPU path: one P976 Encaps and then its Decaps
    per call (count = 1, CUDA-core kernels, the key bound as in the batched
    step), back to back on one stream, host wall-clock from the first launch
    to the final synchronisation; the coins are the batched step's, and the
    keys are checked identical to the batched step's."""
    p = kem.params
    ctx = lwe.Ctx(p, max_batch=1, device=kem.dev.index)
    ctx.set_path(lwe.PATH_SKINNY)
    ctx.bind_key(kem.pk, kem.sk, kem.A)
    pairs = min(pairs, kem.count)
    ct = ctx.empty_ct(pairs)
    K = torch.empty((pairs, 32), dtype=torch.uint8, device=kem.dev)
    K2 = torch.empty_like(K)

    def run(m):
        for i in range(m):
            ctx.encaps(kem.pk, kem.coins[i:i + 1], ct[i:i + 1], K[i:i + 1], A=kem.A)
            ctx.decaps(kem.sk, ct[i:i + 1], K2[i:i + 1], A=kem.A)

    run(16)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(pairs)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    same = torch.equal(K, kem.K[:pairs]) and torch.equal(K2, K) and torch.equal(ct, kem.ct[:pairs])
    ctx.close()
    return pairs / el, bool(same), pairs


# ----------------------------------------------------------------- ours ---
def keccak_perms(length: int, chunk: int = 1024) -> int:
    """Keccak-f[1600] calls of the tree hash of `length` bytes: SHA3-256 of
    each chunk, then of the concatenated 32-byte chunk digests (rate 136
    bytes with at least one padding byte)."""
    full, last = divmod(length, chunk)
    per = lambda L: L // 136 + 1
    leaves = full + (1 if last else 0)
    return full * per(chunk) + (per(last) if last else 0) + per(32 * leaves)


# Derived peaks of the integer-bound kernels at the 2070 MHz maximum SM clock:
#  AES round tables: 160 conflict-free shared-memory lookups per 16-byte block,
#    32 per clock per SM  ->  152 * 2.07e9 * 32 / 160 * 16 B = 1006 GB/s.
#    k_noise's runs of 128 counter blocks share their first two rounds: 133
#    lookups per block, plus the window's 27, worked out for 32 runs at once
#    (one per lane): 27 / (32 x 4) per block -> 133.21 per block -> 1209 GB/s
#  Keccak-f[1600] on 32-bit lanes: 190 integer-ALU operations per round
#    (three-input XORs / chi as LOP3, 64-bit rotations as funnel-shift pairs),
#    64 ALU lanes per clock per SM  ->  152 * 2.07e9 * 64 / (190 * 24)
#    = 4.42 G permutations/s
AES_RUN_PEAK_GBS = 152 * 2.070e9 * 32 / (133 + 27 / 128) * 16 / 1e9
KECCAK_PEAK_GPERMS = 152 * 2.070e9 * 64 / (190 * 24) / 1e9


def algorithmic_bytes(p, count):
    """Bytes each kernel must move through HBM in one step (summed over its
    launches), to set against the measured DRAM traffic."""
    n = p.n
    ct_bytes = 16 * n + 128
    rows = 8 * count
    return {
        # the batched launches: H(c) read in Encaps and in Decaps (H(pk), one
        # message, runs as k_tree_warp)
        "k_tree": float(2 * count * ct_bytes),
        # per launch: S' (bf16) + limbs + E' read; ct written (Encaps) or read (Decaps)
        "k_gemm_tc": 2.0 * (2 * rows * n + 2 * 2 * (n + 8) * n + rows * n + count * ct_bytes),
        # per launch: S' (bf16), E' (int8), E'' written
        "k_noise": 2.0 * count * (2 * 8 * n + 8 * n + 64),
    }


# What bounds each kernel in ncu (profiles/): "alu" above means an
# instruction-throughput bound measured against lwe_probe, not HBM or tensor
LIMITER = {
    "k_noise": "shared-memory pipe: AES round-table lookups plus the sampler's table",
    "k_tree": "integer ALU pipe: Keccak-f XORs, rotations and chi; the balanced schedule "
              "(k_tree_bal) hands SM sub-partition 0's leaves to helper warps after 6 of 8 "
              "permutations and absorbs the roots in two stages: about 33 warp-permutations "
              "on the critical path against 29 of work",
    "k_gemm_tc": "tensor pipe (bf16 tcgen05, CTA pairs)",
}


def algorithmic(p, count):
    """Algorithmic work of the kernels in one step (summed over launches)."""
    n = p.n
    rows, ncols = 8 * count, n + 8
    ct_bytes = 16 * n + 128
    return {
        # two limbs, 2 flops per multiply-add, Encaps + Decaps
        "k_gemm_tc": ("tensor", 2 * (2.0 * 2 * rows * ncols * n), "TFLOP/s", 1e12),
        # AES keystream bytes: S', E' (8n samples each) and E'' (64) per item,
        # 2 bytes per sample, Encaps + Decaps
        "k_noise": ("alu", 2 * (2.0 * (16 * n + 64) * count), "GB/s of AES keystream", 1e9),
        # Keccak-f calls of the batched launches: H(c) in Encaps and in
        # Decaps, and Encaps' K = H(K' || H(c))
        "k_tree": ("alu", float(2 * count * keccak_perms(ct_bytes) + count), "G Keccak-f/s", 1e9),
    }


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a step's
# launches of a kernel, from one ncu capture of this workload (the capture
# and its command are summarised in the named profile).  Each entry carries a
# fingerprint of the source it was measured on: once that source changes the
# figure no longer describes the kernel and the bench reports null.
CSRC = os.path.join(ROOT, "paper_2606_01211_gb300", "csrc")
TRAFFIC = {
    # kernel: (bytes per step, launches per step, [(file, function or None)], fingerprint, profile)
    "k_tree": (129.280000e6, 2,
               [("kem_kernels.cu", "k_tree_bal"), ("kem_kernels.cu", "launch_tree"),
                ("keccak.cuh", None)],
               "61a10e1e45bb906c", "profiles/k_tree_p976.md"),
    "k_gemm_tc": (295.779584e6, 2, [("gemm_tc.cu", None)], "10f4eabbb5ca2195",
                  "profiles/k_gemm_sa2_p976.md"),
    "k_noise": (69.913344e6, 2,
                [("kem_kernels.cu", "k_noise"), ("kem_kernels.cu", "noise_runs"),
                 ("kem_kernels.cu", "noise_store"),
                 ("kem_kernels.cu", "noise_fill_table"), ("kem_kernels.cu", "launch_noise"),
                 ("aes.cuh", None)],
                "8c69346ce7bf41c6", "profiles/k_noise_p976.md"),
}


def _function_text(text: str, name: str) -> str:
    """The source of the first function whose signature line names `name(`,
    up to its closing brace in column 0."""
    i = text.find(" %s(" % name)
    if i < 0:
        return ""
    start = text.rfind("\n", 0, i) + 1
    end = text.find("\n}\n", i)
    return text[start:end + 3] if end >= 0 else text[start:]


def source_fingerprint(parts) -> str:
    import hashlib
    h = hashlib.sha256()
    for fname, func in parts:
        with open(os.path.join(CSRC, fname)) as f:
            text = f.read()
        h.update((_function_text(text, func) if func else text).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel: str):
    """Measured DRAM bytes per launch, or None when unmeasured or stale."""
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    bytes_step, launches, parts, fp, _profile = t
    try:
        if source_fingerprint(parts) != fp:
            return None
    except OSError:
        return None
    return bytes_step / launches


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (whole-job time of independent replicas)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank: int) -> tuple:
    """Each rank is an independent replica with its own key and coins."""
    return 1 + rank, 7 + rank


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2606_01211_gb300 import batch, lwe

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pk_d, _ = peaks()
    p = lwe.Params(**PRESETS[PRESET])
    tuned = batch.autotune(PRESET, COUNT)
    nsteps = args.warmup + args.steps
    key_seed, coin_seed = replica_seeds(rank)
    cs_all = torch.from_numpy(coins(COUNT * nsteps, seed=coin_seed)).to(dev).view(nsteps, COUNT, 32)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    # the step: 4096 Encaps + 4096 Decaps against one key (direct launches,
    # CUDA events around every kernel on its launch stream)
    kem = batch.BatchedKem(PRESET, COUNT, seed=key_seed, gemm_bn=tuned["gemm_bn"],
                           gemm_pair=tuned["gemm_pair"])
    for i in range(args.warmup):
        kem.coins.copy_(cs_all[i])
        kem.step()
    torch.cuda.synchronize()
    assert torch.equal(kem.K, kem.K2), "decapsulated keys differ from the encapsulated keys"

    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        dist.barrier()

    # (1) direct launches with CUDA events around every kernel on its launch
    # stream: the per-kernel times of the roofline.  The side-stream work
    # runs on the main stream here, so that each kernel's events time it
    # alone rather than sharing the GPU with the other stream.
    torch.cuda.synchronize()
    kem.ctx.set_option(lwe.OPT_SERIAL, 1)
    kem.ctx.set_option(lwe.OPT_TIMING, 1)
    kem.ctx.reset_stats()
    evs = []
    for i in range(args.warmup, nsteps):
        flush.fill_(i)  # L2 flush, outside the timed events
        kem.coins.copy_(cs_all[i])
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kem.step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    direct_ms = sum(a.elapsed_time(b) for a, b in evs)
    stats = kem.ctx.kernel_stats()
    kem.ctx.set_option(lwe.OPT_TIMING, 0)
    kem.ctx.set_option(lwe.OPT_SERIAL, 0)
    assert torch.equal(kem.K, kem.K2), "decapsulated keys differ from the encapsulated keys"
    if dist is not None:
        direct_ms = max_over_ranks(direct_ms, dist, dev)
    serial_value = world * COUNT * args.steps / (direct_ms / 1e3)

    # (2) the timed region: the step captured once as a CUDA graph (the
    # workload is defined graph-captured) and replayed with each step's
    # coins; W untimed replays, then K timed ones between barriers
    kem.capture()
    for i in range(args.warmup):
        kem.replay(cs_all[i])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = kem.ctx.launches()
    clk = ClockSampler(local_rank, period_ms=50)
    clk.start(wait_first=True)
    t_region0 = time.time()
    evs = []
    for i in range(args.warmup, nsteps):
        flush.fill_(i)  # L2 flush, outside the timed events
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kem.replay(cs_all[i])
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    t_region1 = time.time()
    clocks = clk.stop(t_region0, t_region1)
    tot_ms = sum(a.elapsed_time(b) for a, b in evs)
    # kernels launched by the replays (the graph's nodes, counted at capture)
    launches = kem.launches_per_step * args.steps + (kem.ctx.launches() - launches0)
    if dist is not None:
        tot_ms = max_over_ranks(tot_ms, dist, dev)
        dist.barrier()
    ok = torch.equal(kem.K, kem.K2)
    err = kem.ctx.device_error()
    value = world * COUNT * args.steps / (tot_ms / 1e3)

    # (3) end to end through the public API: each step's coins from pinned
    # host memory into the graph's input buffer, the replayed step, both key
    # sets back to pinned host memory, all inside the host-timed region
    e2e = None
    if not args.no_e2e:
        hc = torch.from_numpy(coins(COUNT, seed=99)).pin_memory()
        hK = torch.empty((COUNT, 32), dtype=torch.uint8).pin_memory()
        hK2 = torch.empty_like(hK).pin_memory()
        ts = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kem.replay(hc)
            hK.copy_(kem.K, non_blocking=True)
            hK2.copy_(kem.K2, non_blocking=True)
            torch.cuda.synchronize()
            if i >= args.warmup:
                ts.append(time.perf_counter() - t0)
        assert torch.equal(hK, hK2)
        t_e2e = sum(ts)
        if dist is not None:
            t_e2e = max_over_ranks(t_e2e, dist, dev)
        e2e = {"value": world * COUNT * len(ts) / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": COUNT * 32, "d2h_bytes_per_step": 2 * COUNT * 32}

    if rank != 0:
        kem.close()
        return 0

    # roofline of the dominant kernel (largest share of the step): its
    # algorithmic work over the direct-launch steps / its summed event time;
    # the same for each of the three large kernels in `rooflines`
    kernel_total = {k: v[1] for k, v in stats.items()}
    dom = max(kernel_total, key=kernel_total.get)
    alg = algorithmic(p, COUNT)
    probe = None
    if any(alg[k][0] == "alu" for k in alg if k in stats):
        probe = probe_peaks(torch, stream)

    def roof_of(kern):
        bound, work, unit, scale = alg[kern]
        nl, ms_tot = stats[kern]
        ach = work * args.steps / (ms_tot / 1e3) / scale
        if bound == "tensor":
            peak = pk_d.get("bf16_tflops_sustained", pk_d["bf16_tflops"])
        elif kern == "k_noise":
            peak = AES_RUN_PEAK_GBS
        else:
            peak = KECCAK_PEAK_GPERMS
        mp = None
        if bound == "alu" and probe is not None:
            m = probe["aes_run_gbs"] if kern == "k_noise" else probe["keccak_gperms"]
            mp = {"peak": m, "frac": ach / m, "unit": unit,
                  "how": "lwe_probe: the kernel's instruction sequence without memory traffic, "
                         "best of 3 launches; 'peak' is the figure derived from unit counts "
                         "at the maximum SM clock"}
        return {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                "measured_peak": mp,
                "kernel": kern, "launches_per_step": nl / args.steps,
                "share": kernel_total[kern] / sum(kernel_total.values()),
                "algorithmic_bytes": algorithmic_bytes(p, COUNT).get(kern, 0.0) / (nl / args.steps),
                "traffic": traffic_per_launch(kern),
                "timing": "CUDA events around each launch of direct-launch steps, one stream",
                "limiter": LIMITER.get(kern)}

    roof = roof_of(dom) if dom in alg else None
    rooflines = {k: roof_of(k) for k in alg if k in stats}

    # the per-GPU extras (energy, plain path, serving, latency, sweeps, the
    # CPU baseline) are measured at N = 1; a multi-GPU run reports the
    # replicas' throughput only, so the other GPUs are not held meanwhile
    extras = world == 1
    energy = energy_measure(kem, torch, stream, local_rank) if extras and not args.no_energy else None

    # the same 4096-item step with direct launches (no graph) on the
    # CUDA-core product instead of the tensor cores (still one batched call
    # per operation)
    def direct_rate(path):
        kem.ctx.set_path(path)
        for i in range(2):
            kem.step()
        torch.cuda.synchronize()
        ts = []
        for i in range(3):
            flush.fill_(i)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kem.step()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        kem.ctx.set_path(lwe.PATH_TENSOR)
        return COUNT / (statistics.median(ts) / 1e3)

    cuda_core = direct_rate(lwe.PATH_SKINNY) if extras and not args.no_plain else None
    # the last graph replay left the batched results of cs_all[-1] in place
    per_req = None
    if extras and not args.no_plain:
        kem.replay(cs_all[nsteps - 1])
        torch.cuda.synchronize()
        rate, same, m = per_request_rate(kem, lwe, torch, stream)
        per_req = {"value": rate, "unit": UNIT, "pairs": m, "identical_to_batched": same,
                   "how": "one Encaps and its Decaps per call (count = 1, CUDA-core path), "
                          "back to back on one stream, host wall-clock"}
    kem.close()

    served = serve_measure(torch) if extras and not args.no_serve else None
    latency = single_request_latency(lwe, torch, dev) if extras and not args.no_latency else None
    latency_1344 = (single_request_latency(lwe, torch, dev, name="P1344")
                    if extras and not args.no_latency else None)
    sweep = kernel_sweep(lwe, torch, dev, flush) if extras and not args.no_sweep else None
    large = large_n(lwe, torch, dev, batch=args.large_batch) if extras and not args.no_large else None
    ppr = paper_profile(lwe, torch, dev, cpu=not args.no_cpu) if extras and not args.no_pp else None

    cpu = None
    if extras and not args.no_cpu:
        rate, threads, pairs, el = cpu_oracle_rate(target_s=args.cpu_s)
        rate1, _, pairs1, el1 = cpu_oracle_rate(target_s=args.cpu_s / 3, single_thread=True)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d Encaps+Decaps pairs of the P976 workload (A given), %.1f s" % (pairs, el),
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": "%d pairs, %.1f s" % (pairs1, el1)},
               "large_n": None if args.no_large else cpu_large_n(threads)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic (seeded random keys and coins)",
        "config": {"workload": WORKLOAD, "n": p.n, "batch": COUNT, "path": "tensor",
                   "launch": "CUDA graph replay of the captured step",
                   "l2": "flushed between timed steps (256 MiB write), per-step CUDA events",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gpu_launches": launches,
        "roofline": roof,
        "rooflines": rooflines,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "serial_timed_value": serial_value,
        "per_request": per_req,
        "batched_vs_per_request": (value / world / per_req["value"]) if per_req else None,
        "cuda_core_batched_value": cuda_core,
        "batched_vs_cuda_core_batched": (value / world / cuda_core) if cuda_core else None,
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in stats.items()},
        "autotune": {"gemm_pair": tuned["gemm_pair"], "gemm_bn": tuned["gemm_bn"],
                     "tensor_min": tuned["tensor_min"]},
        "energy": energy,
        "served": served,
        "latency_p640_us": latency,
        "latency_p1344_us": latency_1344,
        "as_gbs": sweep["AS_stored"] if sweep else None,
        "kernel_sweep": sweep,
        "large_n": large,
        "paper_profile": ppr,
        "correct": bool(ok) and err == 0,
    }
    print(json.dumps(line))
    return 0


def probe_peaks(torch, stream):
    """Practical peaks of the two integer-bound instruction sequences on
    this GPU: Keccak-f[1600] in registers (k_tree's permutation) and AES
    counter blocks with the shared-memory round tables, in runs whose first
    two rounds are shared (k_noise's generator), no memory traffic
    (lwe_probe).  Best of three launches."""
    from paper_2606_01211_gb300 import lwe
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {}
    for kind, ctas, threads, iters, scale, key in (
            (lwe.PROBE_KECCAK, 3 * sms, 256, 512, 1e9, "keccak_gperms"),
            (lwe.PROBE_AES_RUN, sms, 512, 16384, 1e9 / 16, "aes_run_gbs")):
        sink = torch.empty(ctas * 512, dtype=torch.int32, device="cuda")
        lwe.probe(kind, ctas, iters, sink, stream)
        ts = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lwe.probe(kind, ctas, iters, sink, stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        out[key] = ctas * threads * iters / min(ts) / scale
    return out


def energy_measure(kem, torch, stream, local_rank: int, seconds: float = 3.0):
    """Energy to solution of the step: the captured graph replayed back to
    back for a few seconds while nvidia-smi samples board power every 100 ms;
    energy = mean power x elapsed time (the samples integrated at a uniform
    period), reported per step and as pairs per joule."""
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    for _ in range(20):
        kem.replay()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 0
    clk = ClockSampler(local_rank, period_ms=100)
    clk.start()
    a.record(stream)
    while time.perf_counter() - t0 < seconds:
        for _ in range(100):
            kem.replay()
        steps += 100
        torch.cuda.synchronize()
    b.record(stream)
    torch.cuda.synchronize()
    info = clk.stop()
    watts = getattr(clk, "watts", [])
    if not watts:
        return None
    el = a.elapsed_time(b) / 1e3
    p_avg = statistics.mean(watts)
    pairs = steps * kem.count
    return {"mean_board_w": p_avg, "samples": len(watts), "seconds": el, "steps": steps,
            "joules_per_step": p_avg * el / steps, "pairs_per_joule": pairs / (p_avg * el),
            "sm_mhz": info.get("sm_mhz"), "reasons": info.get("reasons")}


def serve_measure(torch, rates=(1e3, 1e4, 1e5, 1e6), requests: int = 20000):
    """The served mix (KeyGen/Encaps/Decaps 10/70/20 over n in {640, 976,
    1344, 4096}, 10 000 resident keys, Zipf 1.1) over open-loop arrival
    rates, continuous batching versus one launch per request (each run about
    two seconds of arrivals at the low rates, at most `requests`)."""
    from paper_2606_01211_gb300 import serve
    base = serve.ServeConfig(requests=requests)
    store = serve.KeyStore(base, torch.device("cuda", torch.cuda.current_device()))
    sweep = []
    for rate in rates:
        row = {"rate": rate}
        for plain in (False, True):
            cap = 8000 if plain else requests
            c = serve.ServeConfig(**{**base.__dict__, "rate": rate, "plain": plain,
                                     "requests": min(cap, max(2000, int(rate * 2)))})
            eng = serve.Engine(c, store=store)
            eng.warmup()
            st = eng.run()
            row["plain" if plain else "batched"] = {k: st[k] for k in
                                                   ("ops_per_s", "p50_ms", "p99_ms", "mean_batch",
                                                    "requests", "gpu_busy", "tensor_batches",
                                                    "host_launch_s", "makespan_s")}
        row["served_vs_plain"] = row["batched"]["ops_per_s"] / row["plain"]["ops_per_s"]
        sweep.append(row)
    out = dict(next(r for r in sweep if r["rate"] == 1e5)) if 1e5 in rates else dict(sweep[-1])
    out["rate_sweep"] = sweep
    return out


def single_request_latency(lwe, torch, dev, reps: int = 300, name: str = "P640"):
    """One KeyGen, Encaps, Decaps per call (stored A), host wall-clock per
    call including the synchronisation: p50 / p99 in microseconds."""
    p = lwe.Params(**PRESETS[name])
    ctx = lwe.Ctx(p, max_batch=1, device=dev.index)
    ctx.set_path(lwe.PATH_SKINNY)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device=dev)
    ms = torch.from_numpy(master_seeds(reps, seed=5)).to(dev)
    cs = torch.from_numpy(coins(reps, seed=5)).to(dev)
    ct = ctx.empty_ct(1)
    K = torch.empty((1, 32), dtype=torch.uint8, device=dev)
    K2 = torch.empty_like(K)
    t = {"keygen": [], "encaps": [], "decaps": [], "cycle": []}
    torch.cuda.synchronize()
    for i in range(reps):
        t0 = time.perf_counter()
        ctx.keygen(ms[i:i + 1], pk, sk, A_out=A)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.encaps(pk, cs[i:i + 1], ct, K, A=A)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ctx.decaps(sk, ct, K2, A=A)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        if i >= 20:
            t["keygen"].append(t1 - t0)
            t["encaps"].append(t2 - t1)
            t["decaps"].append(t3 - t2)
            t["cycle"].append(t3 - t0)
    assert torch.equal(K, K2)
    # the same Encaps / Decaps against a key bound once (H(pk) not redone)
    t["encaps_bound"], t["decaps_bound"] = [], []
    ctx.bind_key(pk, sk, A)
    torch.cuda.synchronize()
    for i in range(reps):
        t1 = time.perf_counter()
        ctx.encaps(pk, cs[i:i + 1], ct, K, A=A)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ctx.decaps(sk, ct, K2, A=A)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        if i >= 20:
            t["encaps_bound"].append(t2 - t1)
            t["decaps_bound"].append(t3 - t2)
    assert torch.equal(K, K2)
    ctx.close()
    return {k: {"p50": float(np.percentile(v, 50) * 1e6), "p99": float(np.percentile(v, 99) * 1e6)}
            for k, v in t.items()}


def _event_ms(torch, stream, fn, flush=None, reps: int = 5) -> float:
    """Median CUDA-event time of fn() on the stream (after one untimed
    call); L2 flushed before every call when a flush buffer is given."""
    ts = []
    for r in range(reps + 1):
        if flush is not None:
            flush.fill_(r)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        if r:
            ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def kernel_sweep(lwe, torch, dev, flush, sizes=(1344, 2048, 4096, 8192)):
    """Standalone hot kernels over n (L2 flushed before every timed call):
    lwe_expand_A (bytes of A written per second), and lwe_matmul_modq A S
    and S A for one n x 8 secret with A stored (bytes of A read per second)
    or regenerated inside the kernel (bytes of A's keystream per second)."""
    out = {k: {} for k in ("expand_A", "AS_stored", "AS_fused", "SA_stored", "SA_fused")}
    stream = torch.cuda.current_stream()
    for n in sizes:
        A = torch.empty((n, n), dtype=torch.int16, device=dev)
        seed = torch.arange(16, dtype=torch.uint8, device=dev)
        St = torch.randint(-6, 7, (8, n), dtype=torch.int8, device=dev)
        o_as = torch.empty((n, 8), dtype=torch.int16, device=dev)
        o_sa = torch.empty((8, n), dtype=torch.int16, device=dev)
        gb = 2.0 * n * n / 1e9
        out["expand_A"][str(n)] = gb / (_event_ms(torch, stream, lambda: lwe.expand_A(seed, n, 16, A),
                                                  flush) / 1e3)
        out["AS_stored"][str(n)] = gb / (_event_ms(
            torch, stream, lambda: lwe.matmul_modq(lwe.SIDE_AS, St, o_as, n, 16, A=A), flush) / 1e3)
        out["AS_fused"][str(n)] = gb / (_event_ms(
            torch, stream, lambda: lwe.matmul_modq(lwe.SIDE_AS, St, o_as, n, 16, seedA=seed), flush) / 1e3)
        out["SA_stored"][str(n)] = gb / (_event_ms(
            torch, stream, lambda: lwe.matmul_modq(lwe.SIDE_SA, St, o_sa, n, 16, A=A), flush) / 1e3)
        out["SA_fused"][str(n)] = gb / (_event_ms(
            torch, stream, lambda: lwe.matmul_modq(lwe.SIDE_SA, St, o_sa, n, 16, seedA=seed), flush) / 1e3)
        del A
    out["unit"] = "GB/s (bytes of A written, read or generated)"
    return out


# The paper's own timings of this profile (Tab. 2 of the paper: OpenACC on
# one GH200, microseconds per call), for context beside ours
PAPER_PP_US = {1024: (3636.0, 8121.1, 5785.05), 4096: (8576.53, 19668.7, 10551.8)}


def paper_profile(lwe, torch, dev, cpu: bool = True,
                  names=("PP1024", "PP4096", "PP8192", "PP32768")):
    """The paper's own parameter profile (Tab. 1: odd q, one Regev
    encryption per message bit): one KeyGen, Encaps and Decaps per call with
    A stored, CUDA-event ms per call (median of 3), Encaps+Decaps pairs/s,
    and the rate of Encrypt's 256 x n by n x n product (G multiply-adds/s).
    The oracle (numpy, BLAS) is timed on one PP1024 Encaps + Decaps."""
    stream = torch.cuda.current_stream()
    res = {}
    for name in names:
        p = lwe.PpParams(name)
        n = p.n
        ctx = lwe.PpCtx(p, device=dev.index)
        pk, sk, A, ct = ctx.empty_pk(), ctx.empty_sk(), ctx.empty_A(), ctx.empty_ct()
        K = torch.empty(32, dtype=torch.uint8, device=dev)
        K2 = torch.empty_like(K)
        ms = torch.from_numpy(master_seeds(1, seed=11)[0].copy()).to(dev)
        cs = torch.from_numpy(coins(1, seed=11)[0].copy()).to(dev)
        kg = _event_ms(torch, stream, lambda: ctx.keygen(ms, pk, sk, A), None, reps=3)
        en = _event_ms(torch, stream, lambda: ctx.encaps(pk, A, cs, ct, K), None, reps=3)
        de = _event_ms(torch, stream, lambda: ctx.decaps(sk, A, ct, K2), None, reps=3)
        torch.cuda.synchronize()
        assert torch.equal(K, K2)
        # the same calls against the bound key (H(pk) and A's limbs once)
        ctx.bind_key(pk, A)
        enb = _event_ms(torch, stream, lambda: ctx.encaps(pk, A, cs, ct, K), None, reps=3)
        deb = _event_ms(torch, stream, lambda: ctx.decaps(sk, A, ct, K2), None, reps=3)
        torch.cuda.synchronize()
        assert torch.equal(K, K2)
        ctx.bind_key()
        r = {"keygen_ms": kg, "encaps_ms": en, "decaps_ms": de,
             "encaps_bound_ms": enb, "decaps_bound_ms": deb,
             "pairs_per_s": 1e3 / (en + de), "pairs_per_s_bound": 1e3 / (enb + deb),
             "encrypt_gmac_per_s": 256.0 * n * n / (en / 1e3) / 1e9,
             "ct_bytes": p.ct_bytes}
        if n in PAPER_PP_US:
            pk_, pe, pd = PAPER_PP_US[n]
            r["paper_gh200_ms"] = {"keygen": pk_ / 1e3, "encaps": pe / 1e3, "decaps": pd / 1e3}
            r["encaps_decaps_vs_paper"] = (pe + pd) / 1e3 / (en + de)
        res[name] = r
        ctx.close()
        del A
    if cpu:
        from oracle import pp as opp
        po = opp.preset("PP1024")
        pk_o, sk_o, A_o = opp.keygen(po, bytes(32), want_A=True)
        t0 = time.perf_counter()
        ct_o, _ = opp.encaps(po, pk_o, bytes(range(32)), A_o)
        opp.decaps(po, sk_o, ct_o, A_o)
        res["oracle_PP1024_encaps_decaps_ms"] = (time.perf_counter() - t0) * 1e3
    res["unit"] = "ms per call; one item per call"
    return res


def large_n(lwe, torch, dev, batch: int = 1024, names=("P16384", "P32768")):
    """n = 16384 and 32768 (A = 0.5 / 2 GiB): one KeyGen, Encaps and Decaps
    per call with A stored in HBM vs regenerated tile by tile inside the
    kernels (CUDA-core path), and Encaps of `batch` items against one key
    on the tensor path (K split into exact passes).  CUDA-event ms per call
    (median of 3); the batched figure also as Encaps/s."""
    stream = torch.cuda.current_stream()
    res = {}
    for name in names:
        p = lwe.Params(**PRESETS[name])
        n = p.n
        ctx = lwe.Ctx(p, max_batch=batch, device=dev.index)
        ms = torch.from_numpy(master_seeds(1, seed=3)).to(dev)
        cs = torch.from_numpy(coins(batch, seed=3)).to(dev)
        pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
        A = torch.empty((n, n), dtype=torch.int16, device=dev)
        ct = ctx.empty_ct(batch)
        K = torch.empty((batch, 32), dtype=torch.uint8, device=dev)
        K2 = torch.empty_like(K)
        r = {}
        ctx.set_path(lwe.PATH_SKINNY)
        for mode, Ak in (("stored", A), ("fused", None)):
            r["keygen_" + mode] = _event_ms(torch, stream, lambda: ctx.keygen(ms, pk, sk, A_out=Ak),
                                            reps=3)
            r["encaps_" + mode] = _event_ms(torch, stream, lambda: ctx.encaps(pk, cs[:1], ct[:1], K[:1],
                                                                               A=Ak), reps=3)
            r["decaps_" + mode] = _event_ms(torch, stream, lambda: ctx.decaps(sk, ct[:1], K2[:1], A=Ak),
                                            reps=3)
            assert torch.equal(K[:1], K2[:1])
        ctx.keygen(ms, pk, sk, A_out=A)
        ctx.set_path(lwe.PATH_TENSOR)
        t = _event_ms(torch, stream, lambda: ctx.encaps(pk, cs, ct, K, A=A), reps=3)
        r["encaps_batched_%d_stored" % batch] = t
        r["encaps_batched_per_s"] = batch / (t / 1e3)
        r["encaps_batched_kernels"] = batched_kernels(lwe, torch, ctx, n, batch,
                                                      lambda: ctx.encaps(pk, cs, ct, K, A=A))
        # the same calls against a bound key (H(pk) and the limbs of [A | B]
        # made once, as a server holding the key does)
        ctx.bind_key(pk, sk, A)
        tb = _event_ms(torch, stream, lambda: ctx.encaps(pk, cs, ct, K, A=A), reps=3)
        r["encaps_batched_%d_bound" % batch] = tb
        r["encaps_batched_bound_per_s"] = batch / (tb / 1e3)
        r["encaps_batched_bound_kernels"] = batched_kernels(
            lwe, torch, ctx, n, batch, lambda: ctx.encaps(pk, cs, ct, K, A=A))["ms"]
        ctx.bind_key(None)
        ctx.decaps(sk, ct, K2, A=A)
        torch.cuda.synchronize()
        assert torch.equal(K, K2)
        r["row_split"] = row_split_times(lwe, torch, stream, A, n)
        res[name] = r
        ctx.close()
        del A
        torch.cuda.empty_cache()
    res["unit"] = "ms per call"
    return res


def batched_kernels(lwe, torch, ctx, n, batch, call):
    """Per-kernel split of one batched call (CUDA events around each launch,
    side-stream work on the caller's stream) and the rate of its tensor-core
    GEMM: 2 limbs x 2 flops x (8 batch) rows x (n + 8) columns x n, over the
    GEMM's K-split launches, against the bf16 burst peak (MEASURED_PEAKS.json,
    else the fallback figure)."""
    ctx.set_option(lwe.OPT_TIMING, 1)
    ctx.set_option(lwe.OPT_SERIAL, 1)
    ctx.reset_stats()
    call()
    torch.cuda.synchronize()
    ks = ctx.kernel_stats()
    ctx.set_option(lwe.OPT_TIMING, 0)
    ctx.set_option(lwe.OPT_SERIAL, 0)
    out = {"ms": {k: round(v[1], 4) for k, v in ks.items()},
           "launches": {k: v[0] for k, v in ks.items()}}
    g = ks.get("k_gemm_tc")
    if g and g[1] > 0:
        tflops = 4.0 * 8 * batch * (n + 8) * n / (g[1] * 1e-3) / 1e12
        pk, how = peaks()
        out["gemm_tflops"] = tflops
        out["gemm_frac_of_bf16_burst"] = tflops / pk["bf16_tflops"]
        out["peak_source"] = how
    return out


def row_split_times(lwe, torch, stream, A, n, worlds=(2, 4)):
    """One GPU's share of a row-split product (lwe_matmul_modq_rows over rank
    0's block of rows, A stored or regenerated) against the whole product on
    one GPU, CUDA-event ms (median of 3).  The collectives (an all-gather of
    16 n bytes, a sum-reduction of 32 n bytes) are not timed here: every run
    of this benchmark has one GPU."""
    from paper_2606_01211_gb300 import rowsplit
    dev = A.device
    St = torch.randint(-6, 7, (8, n), dtype=torch.int8, device=dev)
    seed = torch.arange(16, dtype=torch.uint8, device=dev)
    o_as = torch.empty((n, 8), dtype=torch.int16, device=dev)
    o_sa = torch.empty((8, n), dtype=torch.int16, device=dev)
    out = {}
    for world in (1,) + tuple(worlds):
        r0, r1 = rowsplit.row_block(n, world, 0)
        blk = A[r0:r1]
        t = {}
        for mode, Ar, sd in (("stored", blk, None), ("fused", None, seed)):
            t["AS_" + mode] = _event_ms(torch, stream, lambda: lwe.matmul_modq_rows(
                lwe.SIDE_AS, St, o_as, n, 16, r0, r1, A_rows=Ar, seedA=sd), reps=3)
            t["SA_" + mode] = _event_ms(torch, stream, lambda: lwe.matmul_modq_rows(
                lwe.SIDE_SA, St, o_sa, n, 16, r0, r1, A_rows=Ar, seedA=sd), reps=3)
        out["world%d_rank0" % world] = t
    out["unit"] = "ms per call on one GPU (its rows only)"
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-energy", action="store_true")
    ap.add_argument("--no-pp", action="store_true")
    ap.add_argument("--sweep-only", type=str, default=None, metavar="N[,N...]",
                    help="only the standalone kernel sweep at these n (prints its JSON, not the bench line)")
    ap.add_argument("--large-only", type=str, default=None, metavar="NAME[,NAME...]",
                    help="only the large-n section for these presets (prints its JSON, not the bench line)")
    ap.add_argument("--pp-only", type=str, default=None, metavar="NAME[,NAME...]",
                    help="only the paper-profile section for these presets, without the oracle (prints its JSON)")
    ap.add_argument("--large-batch", type=int, default=1024,
                    help="Encaps per batched call in the large-n section")
    ap.add_argument("--cpu-s", type=float, default=12.0)
    ap.add_argument("--ref-step-s", type=float, default=None,
                    help="CPU seconds per reference step (default: about 150 s in all)")
    args = ap.parse_args()
    if args.sweep_only:
        import torch
        from paper_2606_01211_gb300 import lwe
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
        sizes = tuple(int(x) for x in args.sweep_only.split(","))
        print(json.dumps(kernel_sweep(lwe, torch, dev, flush, sizes=sizes)))
        return 0
    if args.pp_only:
        import torch
        from paper_2606_01211_gb300 import lwe
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        names = tuple(args.pp_only.split(","))
        print(json.dumps(paper_profile(lwe, torch, dev, cpu=False, names=names)))
        return 0
    if args.large_only:
        import torch
        from paper_2606_01211_gb300 import lwe
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        names = tuple(args.large_only.split(","))
        print(json.dumps(large_n(lwe, torch, dev, batch=args.large_batch, names=names)))
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_ours(args, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
