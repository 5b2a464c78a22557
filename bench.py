"""Benchmark of the batched plain-LWE KEM hot path on GB300.

Workload (one step): one P976 public key (n = 976, q = 2^16, sigma = 2.3,
c = 10, B = 3), 4096 Encaps against it (stacked S' on the tensor-core path)
followed by the 4096 matching Decaps.  Inputs (keys, expanded A, the coins of
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
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ reference ---
def cpu_oracle_rate(target_s: float = 12.0, max_pairs: int | None = None):
    """The plain oracle (as it stands) on all host cores over a bounded
    sample of the workload: Encaps + Decaps pairs per second."""
    from oracle import oracle as O
    cfg = PRESETS[PRESET]
    po = O.Params(**cfg)
    pk, sk, A = O.keygen(po, bytes(master_seeds(1, seed=1)[0]), want_A=True)
    threads = len(os.sched_getaffinity(0))
    threads = min(threads, O.max_threads()) if O.max_threads() > 1 else 1
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


# ----------------------------------------------------------------- ours ---
def algorithmic(p, count):
    """Per-launch algorithmic work of the kernels of one step."""
    n = p.n
    rows, ncols = 8 * count, n + 8
    return {
        # two limbs, 2 flops per multiply-add
        "k_gemm_tc": ("tensor", 2.0 * 2 * rows * ncols * n, "flop"),
        # AES keystream bytes: S', E' (8n samples each) and E'' (64) per item,
        # 2 bytes per sample
        "k_noise": ("alu", 2.0 * (16 * n + 64) * count, "keystream bytes"),
    }


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2606_01211_gb300 import lwe

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pk_d, _ = peaks()
    p = lwe.Params(**PRESETS[PRESET])
    ctx = lwe.Ctx(p, max_batch=COUNT, device=local_rank)
    ctx.set_path(lwe.PATH_TENSOR)
    pk, sk = ctx.empty_pk(1), ctx.empty_sk(1)
    A = torch.empty((p.n, p.n), dtype=torch.int16, device=dev)
    ms = torch.from_numpy(master_seeds(1, seed=1 + rank)).to(dev)
    ctx.keygen(ms, pk, sk, A_out=A)
    nsteps = args.warmup + args.steps
    cs_all = torch.from_numpy(coins(COUNT * nsteps, seed=7 + rank)).to(dev).view(nsteps, COUNT, 32)
    ct = ctx.empty_ct(COUNT)
    K = torch.empty((COUNT, 32), dtype=torch.uint8, device=dev)
    K2 = torch.empty_like(K)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(i):
        ctx.encaps(pk, cs_all[i], ct, K, A=A)
        ctx.decaps(sk, ct, K2, A=A)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    assert torch.equal(K, K2), "decapsulated keys differ from the encapsulated keys"

    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        dist.barrier()
    torch.cuda.synchronize()
    ctx.set_option(lwe.OPT_TIMING, 1)
    ctx.reset_stats()
    launches0 = ctx.launches()
    clk = ClockSampler(local_rank)
    clk.start()
    evs = []
    for i in range(args.warmup, nsteps):
        flush.fill_(i)  # L2 flush, outside the timed events
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(i)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = ctx.launches() - launches0
    stats = ctx.kernel_stats()
    ctx.set_option(lwe.OPT_TIMING, 0)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        dist.barrier()
    ok = torch.equal(K, K2)
    err = ctx.device_error()
    value = world * COUNT * args.steps / (tot_ms / 1e3)

    if rank != 0:
        return 0

    # roofline of the dominant kernel (largest share of the timed region)
    kernel_total = {k: v[1] for k, v in stats.items()}
    dom = max(kernel_total, key=kernel_total.get)
    alg = algorithmic(p, COUNT)
    roof = None
    if dom in alg:
        bound, work, what = alg[dom]
        nl, ms_tot = stats[dom]
        per_launch_ms = ms_tot / nl
        if bound == "tensor":
            ach = work / (per_launch_ms / 1e3) / 1e12
            peak = pk_d.get("bf16_tflops_sustained", pk_d["bf16_tflops"])
            roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak}
        else:
            ach = work / (per_launch_ms / 1e3) / 1e9
            roof = {"bound": "alu", "achieved": ach, "peak": args.aes_peak_gbs,
                    "unit": "GB/s of AES keystream", "frac": ach / args.aes_peak_gbs}
        roof["kernel"] = dom
        roof["share"] = kernel_total[dom] / sum(kernel_total.values())
        roof["traffic"] = None

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hc = torch.from_numpy(coins(COUNT, seed=99)).pin_memory()
        hK = torch.empty((COUNT, 32), dtype=torch.uint8).pin_memory()
        hK2 = torch.empty_like(hK).pin_memory()
        dc = torch.empty((COUNT, 32), dtype=torch.uint8, device=dev)
        ts = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dc.copy_(hc, non_blocking=True)
            ctx.encaps(pk, dc, ct, K, A=A)
            ctx.decaps(sk, ct, K2, A=A)
            hK.copy_(K, non_blocking=True)
            hK2.copy_(K2, non_blocking=True)
            torch.cuda.synchronize()
            if i >= args.warmup:
                ts.append(time.perf_counter() - t0)
        assert torch.equal(hK, hK2)
        e2e = {"value": COUNT / statistics.mean(ts), "unit": UNIT,
               "h2d_bytes_per_step": COUNT * 32, "d2h_bytes_per_step": 2 * COUNT * 32}

    # the plain per-request path (CUDA cores, one item per row of CTAs)
    plain = None
    if not args.no_plain:
        ctx.set_path(lwe.PATH_SKINNY)
        for i in range(2):
            step(i)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(0)
        b.record(stream)
        torch.cuda.synchronize()
        plain = COUNT / (a.elapsed_time(b) / 1e3)
        ctx.set_path(lwe.PATH_TENSOR)

    cpu = None
    if not args.no_cpu:
        rate, threads, pairs, el = cpu_oracle_rate(target_s=args.cpu_s)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d Encaps+Decaps pairs of the P976 workload (A given), %.1f s" % (pairs, el)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic (seeded random keys and coins)",
        "config": {"workload": WORKLOAD, "n": p.n, "batch": COUNT, "path": "tensor",
                   "l2": "flushed between timed steps (256 MiB write), per-step CUDA events",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "plain_path_value": plain,
        "batched_vs_plain": (value / world / plain) if plain else None,
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in stats.items()},
        "correct": bool(ok) and err == 0,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-s", type=float, default=12.0)
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    # AES keystream peak (GB/s): 152 SMs x 2070 MHz x 32 shared-memory
    # lookups per clock / 160 lookups per 16-byte block
    ap.add_argument("--aes-peak-gbs", type=float, default=152 * 2.070e9 * 32 / 160 * 16 / 1e9)
    args = ap.parse_args()

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
