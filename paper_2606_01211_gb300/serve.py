"""Continuous-batching server for the plain-LWE KEM on one GPU.

Requests (KeyGen for a dimension n, Encaps or Decaps against a resident key)
arrive open-loop and queue per (operation, n).  Whenever one of the
engine's slots is free it takes the queue whose head is oldest and launches
ONE batched library call on that slot's stream: all waiting requests of one
key when that key has many (a single-key call, where the stacked S' can use
the tensor-core product), else the oldest requests across keys (a
multi-key call with per-item key pointers).  It does not wait for the
batches already running on the other slots, so arrivals are admitted while
earlier work is still on the device (continuous batching).  Completion is
observed through CUDA events; latency is measured from a request's arrival
to the moment its batch is seen complete.

Keys (pk, sk) stay on the device.  The expanded matrix A of a key is kept
in an LRU cache that grows while the device has free memory: a miss takes a
free slot, else a new chunk of slots when the live free device memory (read
at that moment) stays above a reserve and the byte budget allows, else it
evicts the least recently used A.  A key whose A is not cached is served
with A regenerated inside the kernels from its seed (the paper's on-demand
generation, Sec. 4.3).  A batch of one key (one request at low load, or a
hot key) is one single-key library call; only batches that mix keys take
the per-item key pointers.

The engine only moves buffers and orders calls: every step of KeyGen,
Encaps and Decaps runs in liblwe.so's kernels.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import lwe
from .inputs import PRESETS, coins as make_coins, master_seeds, rng

OPS = ("keygen", "encaps", "decaps")


@dataclass
class ServeConfig:
    presets: tuple = ("P640", "P976", "P1344", "P4096")
    mix: tuple = (0.10, 0.70, 0.20)           # keygen, encaps, decaps
    keys_per_n: int = 2500                     # 10 000 resident keys over 4 n
    zipf_s: float = 1.1
    rate: float = 1e4                          # requests per second
    requests: int = 20000
    max_batch: int = 512
    slots: int = 4
    a_budget_bytes: int | None = None          # None: no cap beyond the live free memory
    reserve_bytes: int = 8 << 30               # free device memory the A cache leaves alone
    seed: int = 1
    plain: bool = False                        # per-request launches (baseline)


@dataclass
class Request:
    rid: int
    op: int                                    # index into OPS
    n: int
    key: int                                   # key index (-1 for keygen)
    t_arr: float
    t_done: float = 0.0


def zipf_keys(count: int, n_keys: int, s: float, r: np.random.Generator) -> np.ndarray:
    w = 1.0 / np.arange(1, n_keys + 1) ** s
    return r.choice(n_keys, size=count, p=w / w.sum())


class KeyStore:
    """Resident key pairs per dimension and an LRU cache of expanded A.

    The cache holds fixed slots of 2 n^2 bytes per dimension, in chunks of
    CHUNK_BYTES.  A miss takes a free slot; with none free, a new chunk is
    allocated if the device's free memory, read live, stays above the
    reserve after it and the byte budget (if any) allows; otherwise the
    least recently used A of that dimension is evicted (a dimension that
    holds no slot then serves the key with A regenerated).  A slot that is
    reused waits, on the stream that refills it, for the last batch that
    read it.  The most popular keys are expanded up front, up to an even
    share per dimension of what the budget or the free memory allows."""

    CHUNK_BYTES = 256 << 20

    def __init__(self, cfg: ServeConfig, device: torch.device, prefill: bool = True):
        self.dev = device
        self.cfg = cfg
        self.params = {}
        self.pk, self.sk = {}, {}
        self.hits = self.misses = self.fills = self.grows = 0
        self.chunks, self.slot_at, self.slot_of, self.lru, self.free, self.last_use = \
            {}, {}, {}, {}, {}, {}
        self.ready = {}
        # vectorised views for batches across keys: the slot of each key
        # (-1: not cached) and the device address of each slot
        self.slot_np, self.slot_ptr, self.ready_done = {}, {}, {}
        self.budget = cfg.a_budget_bytes
        self.reserve = cfg.reserve_bytes
        self.used = 0
        for i, name in enumerate(cfg.presets):
            p = lwe.Params(**PRESETS[name])
            n = p.n
            self.params[n] = p
            ctx = lwe.Ctx(p, max_batch=min(cfg.keys_per_n, 256), device=device.index)
            ms = torch.from_numpy(master_seeds(cfg.keys_per_n, seed=cfg.seed * 100 + i)).to(device)
            pk = torch.empty((cfg.keys_per_n, p.pk_bytes), dtype=torch.uint8, device=device)
            sk = torch.empty((cfg.keys_per_n, p.sk_bytes), dtype=torch.uint8, device=device)
            for a in range(0, cfg.keys_per_n, 256):
                b = min(cfg.keys_per_n, a + 256)
                ctx.keygen(ms[a:b], pk[a:b], sk[a:b])
            self.pk[n], self.sk[n] = pk, sk
            ctx.close()
            self.chunks[n], self.slot_at[n] = [], []
            self.slot_of[n] = {}
            self.lru[n] = collections.OrderedDict()
            self.free[n], self.last_use[n], self.ready[n] = [], [], []
            self.slot_np[n] = np.full(cfg.keys_per_n, -1, np.int64)
            self.slot_ptr[n] = np.zeros(0, np.int64)
            self.ready_done[n] = []
        if prefill:  # key k is the (k+1)-th most popular (Zipf rank)
            share = self._share()
            for n in self.params:
                for k in range(min(cfg.keys_per_n, share // (2 * n * n))):
                    if self._fill(n, k, torch.cuda.current_stream(device)) is None:
                        break
        torch.cuda.synchronize(device)
        self.hits = self.misses = self.fills = 0

    def _share(self) -> int:
        """Each dimension's fair share of the cache: the budget, or what the
        device could hold now above the reserve, split evenly."""
        free, _ = torch.cuda.mem_get_info(self.dev)
        room = self.used + max(0, free - self.reserve)
        if self.budget is not None:
            room = min(room, self.budget)
        return room // max(1, len(self.params))

    def _grow(self, n) -> bool:
        """One more chunk of slots for dimension n, if live free memory and
        the budget allow."""
        slot_bytes = 2 * n * n
        per = max(1, self.CHUNK_BYTES // slot_bytes)
        per = min(per, self.cfg.keys_per_n - len(self.slot_at[n]))
        if per <= 0:
            return False
        nbytes = per * slot_bytes
        if self.budget is not None and self.used + nbytes > self.budget:
            per = (self.budget - self.used) // slot_bytes
            nbytes = per * slot_bytes
            if per <= 0:
                return False
        free, _ = torch.cuda.mem_get_info(self.dev)
        if free - nbytes < self.reserve:
            return False
        chunk = torch.empty((per, n, n), dtype=torch.int16, device=self.dev)
        self.chunks[n].append(chunk)
        base = len(self.slot_at[n])
        for j in range(per):
            self.slot_at[n].append(chunk[j])
            self.last_use[n].append(None)
            self.ready[n].append(None)
            self.ready_done[n].append(False)
        self.slot_ptr[n] = np.concatenate(
            [self.slot_ptr[n], chunk.data_ptr() + 2 * n * n * np.arange(per, dtype=np.int64)])
        self.free[n].extend(range(base + per - 1, base - 1, -1))
        self.used += nbytes
        self.grows += 1
        return True

    def _fill(self, n, key, stream):
        if not self.free[n] and not self._grow(n) and not self.lru[n]:
            return None
        self.fills += 1
        if self.free[n]:
            s = self.free[n].pop()
        else:
            old, s = self.lru[n].popitem(last=False)
            del self.slot_of[n][old]
            self.slot_np[n][old] = -1
            if self.last_use[n][s] is not None:
                stream.wait_event(self.last_use[n][s])
        with torch.cuda.stream(stream):
            lwe.expand_A(self.pk[n][key, :16], n, self.params[n].logq, self.slot_at[n][s],
                         stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.ready[n][s] = ev
        self.ready_done[n][s] = False
        self.slot_of[n][key] = s
        self.slot_np[n][key] = s
        self.lru[n][key] = s
        return s

    def _wait_ready(self, n, s, stream):
        """Order `stream` after the fill of slot s, until that fill is seen
        complete (then no wait is needed any more)."""
        if self.ready_done[n][s]:
            return
        ev = self.ready[n][s]
        if ev.query():
            self.ready_done[n][s] = True
        else:
            stream.wait_event(ev)

    def cached(self, n: int, key: int) -> bool:
        return key in self.slot_of[n]

    def A(self, n: int, key: int, stream: torch.cuda.Stream, admit: bool = True):
        """The cached A of a key (LRU order refreshed), expanding it into a
        free or least recently used slot on a miss; None = regenerate A
        inside the kernels (no slot for this dimension, or admit=False)."""
        s = self.slot_of[n].get(key)
        if s is not None:
            self.lru[n].move_to_end(key)
            self.hits += 1
            self._wait_ready(n, s, stream)  # filled, possibly on another stream
            return self.slot_at[n][s]
        self.misses += 1
        if not admit:
            return None
        s = self._fill(n, key, stream)
        return None if s is None else self.slot_at[n][s]

    def cached_slots(self, n: int, keys: np.ndarray) -> np.ndarray:
        """The slot of each key of a batch (-1: not cached)."""
        return self.slot_np[n][keys]

    def A_ptrs(self, n: int, keys: np.ndarray, stream: torch.cuda.Stream) -> np.ndarray:
        """Device addresses of the cached A of keys that are all cached:
        each distinct key's LRU order refreshed once, each distinct slot's
        fill ordered before `stream` once."""
        slots = self.slot_np[n][keys]
        for k in np.unique(keys).tolist():
            self.lru[n].move_to_end(k)
        for sl in np.unique(slots).tolist():
            self._wait_ready(n, sl, stream)
        self.hits += len(keys)
        return self.slot_ptr[n][slots]

    def used_by(self, n: int, keys, event: torch.cuda.Event):
        """Record the batch that reads these keys' cached A."""
        slots = self.slot_np[n][np.asarray(list(keys), dtype=np.int64)]
        for sl in np.unique(slots[slots >= 0]).tolist():
            self.last_use[n][sl] = event


class Slot:
    """A stream with its own contexts and staging buffers."""

    def __init__(self, store: KeyStore, max_batch: int, device: torch.device, plain: bool):
        self.stream = torch.cuda.Stream(device=device)
        self.ctx, self.buf = {}, {}
        for n, p in store.params.items():
            c = lwe.Ctx(p, max_batch=max_batch, device=device.index)
            c.set_path(lwe.PATH_SKINNY if plain else lwe.PATH_AUTO)
            self.ctx[n] = c
            self.buf[n] = dict(
                seeds=torch.empty((max_batch, 32), dtype=torch.uint8, device=device),
                coins=torch.empty((max_batch, 32), dtype=torch.uint8, device=device),
                ct=torch.empty((max_batch, p.ct_bytes), dtype=torch.uint8, device=device),
                K=torch.empty((max_batch, 32), dtype=torch.uint8, device=device),
                pk=torch.empty((max_batch, p.pk_bytes), dtype=torch.uint8, device=device),
                sk=torch.empty((max_batch, p.sk_bytes), dtype=torch.uint8, device=device))
        # per-item key pointers of a multi-key batch (pinned host -> device)
        self.h_ptr = torch.empty((3, max_batch), dtype=torch.int64).pin_memory()
        self.d_ptr = torch.empty((3, max_batch), dtype=torch.int64, device=device)
        self.event = None
        self.reqs: list = []


class Engine:
    """Open-loop server over pre-generated request payloads."""

    def __init__(self, cfg: ServeConfig, store: KeyStore | None = None, device=None):
        self.cfg = cfg
        self.dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.store = store or KeyStore(cfg, self.dev)
        mb = 1 if cfg.plain else cfg.max_batch
        self.slots = [Slot(self.store, mb, self.dev, cfg.plain) for _ in range(cfg.slots)]
        self.spans = []
        self.n_single = self.n_multi = self.n_tensor = 0
        self._make_requests()

    # ---- workload --------------------------------------------------------
    def _make_requests(self):
        cfg = self.cfg
        # one generator per field, so that a shorter run is a prefix of a
        # longer one with the same seed
        N = cfg.requests
        gaps = rng(cfg.seed + 7).exponential(1.0 / cfg.rate, size=N)
        t_arr = np.cumsum(gaps) - gaps[0]
        ops = rng(cfg.seed + 8).choice(3, size=N, p=np.asarray(cfg.mix) / np.sum(cfg.mix))
        ns = np.array(sorted(self.store.params))
        nsel = ns[rng(cfg.seed + 9).integers(0, len(ns), size=N)]
        keys = zipf_keys(N, cfg.keys_per_n, cfg.zipf_s, rng(cfg.seed + 10))
        self.reqs = [Request(i, int(ops[i]), int(nsel[i]), int(keys[i]) if ops[i] else -1,
                             float(t_arr[i])) for i in range(N)]
        # per-n payload and result pools, indexed by the request id
        self.pool = {}
        for n, p in self.store.params.items():
            idx = [q.rid for q in self.reqs if q.n == n]
            self.pool[n] = dict(row={rid: j for j, rid in enumerate(idx)})
        seeds = master_seeds(N, seed=cfg.seed + 11)
        cns = make_coins(N, seed=cfg.seed + 13)
        dec_coins = make_coins(N, seed=cfg.seed + 17)
        for n, p in self.store.params.items():
            rows = self.pool[n]["row"]
            ids = np.fromiter(rows.keys(), dtype=np.int64, count=len(rows))
            m = max(1, len(ids))
            P = self.pool[n]
            P["seeds"] = torch.from_numpy(seeds[ids] if len(ids) else seeds[:1]).to(self.dev)
            P["coins"] = torch.from_numpy(cns[ids] if len(ids) else cns[:1]).to(self.dev)
            P["ct"] = torch.zeros((m, p.ct_bytes), dtype=torch.uint8, device=self.dev)
            P["K"] = torch.zeros((m, 32), dtype=torch.uint8, device=self.dev)
            P["pk"] = torch.zeros((m, p.pk_bytes), dtype=torch.uint8, device=self.dev)
            P["sk"] = torch.zeros((m, p.sk_bytes), dtype=torch.uint8, device=self.dev)
            # Decaps inputs: ciphertexts made beforehand through the plain path
            P["dct"] = torch.zeros((m, p.ct_bytes), dtype=torch.uint8, device=self.dev)
            P["dK"] = torch.zeros((m, 32), dtype=torch.uint8, device=self.dev)
            dec = [q for q in self.reqs if q.n == n and OPS[q.op] == "decaps"]
            if dec:
                ctx = lwe.Ctx(p, max_batch=1, device=self.dev.index)
                ctx.set_path(lwe.PATH_SKINNY)
                dcs = torch.from_numpy(dec_coins[[q.rid for q in dec]]).to(self.dev)
                for j, q in enumerate(dec):
                    row = rows[q.rid]
                    ctx.encaps(self.store.pk[n][q.key], dcs[j:j + 1], P["dct"][row:row + 1],
                               P["dK"][row:row + 1])
                torch.cuda.synchronize(self.dev)
                ctx.close()

    # ---- serving ---------------------------------------------------------
    HOT = 64          # waiting requests of one key that justify a single-key batch
    ADMIT = 8         # cache misses admitted (A expanded) per dispatch
    TENSOR_MIN = 64   # the contexts' default LWE_OPT_TENSOR_MIN (AUTO path)

    def _key_ptrs(self, n: int, keys: np.ndarray, what: str) -> np.ndarray:
        p = self.store.params[n]
        if what == "pk":
            return self.store.pk[n].data_ptr() + keys * p.pk_bytes
        if what == "sk":
            return self.store.sk[n].data_ptr() + keys * p.sk_bytes
        return self.store.sk[n].data_ptr() + keys * p.sk_bytes + 8 * n + 32  # H(pk) in sk

    def _launch(self, slot: Slot, group: list, single_key: bool):
        q0 = group[0]
        n, op = q0.n, OPS[q0.op]
        P, B, ctx = self.pool[n], slot.buf[n], slot.ctx[n]
        rows = torch.tensor([P["row"][q.rid] for q in group], dtype=torch.long)
        cnt = len(group)
        st = slot.stream
        if op != "keygen":
            if single_key:
                self.n_single += 1
                self.n_tensor += int(cnt >= self.TENSOR_MIN and not self.cfg.plain)
            else:
                self.n_multi += 1
        with torch.cuda.stream(st):
            t_start = torch.cuda.Event(enable_timing=True)
            t_start.record(st)
            rows_d = rows.to(self.dev, non_blocking=True)
            if op == "keygen":
                torch.index_select(P["seeds"], 0, rows_d, out=B["seeds"][:cnt])
                ctx.keygen(B["seeds"][:cnt], B["pk"][:cnt], B["sk"][:cnt], stream=st)
                P["pk"].index_copy_(0, rows_d, B["pk"][:cnt])
                P["sk"].index_copy_(0, rows_d, B["sk"][:cnt])
            elif single_key:
                A = self.store.A(n, q0.key, st)
                if op == "encaps":
                    torch.index_select(P["coins"], 0, rows_d, out=B["coins"][:cnt])
                    ctx.encaps(self.store.pk[n][q0.key], B["coins"][:cnt], B["ct"][:cnt],
                               B["K"][:cnt], A=A, stream=st)
                    P["ct"].index_copy_(0, rows_d, B["ct"][:cnt])
                else:
                    torch.index_select(P["dct"], 0, rows_d, out=B["ct"][:cnt])
                    ctx.decaps(self.store.sk[n][q0.key], B["ct"][:cnt], B["K"][:cnt], A=A,
                               stream=st, count=cnt)
                P["K"].index_copy_(0, rows_d, B["K"][:cnt])
            else:
                # across keys: items whose A is cached, then the others (A
                # regenerated); a few misses are admitted to the cache
                keys = np.fromiter((q.key for q in group), dtype=np.int64, count=cnt)
                cached = self.store.cached_slots(n, keys) >= 0
                admitted = 0
                for k in np.unique(keys[~cached]).tolist():
                    if admitted >= self.ADMIT:
                        break
                    if self.store.A(n, k, st) is not None:
                        admitted += 1
                cached = self.store.cached_slots(n, keys) >= 0
                order = np.concatenate([np.nonzero(cached)[0], np.nonzero(~cached)[0]])
                keys = keys[order]
                rows_o = rows[torch.from_numpy(order)]
                rows_d = rows_o.to(self.dev, non_blocking=True)
                nst = int(cached.sum())
                what = "pk" if op == "encaps" else "sk"
                hp = slot.h_ptr.numpy()
                hp[0, :cnt] = self._key_ptrs(n, keys, what)
                if op == "encaps":
                    hp[1, :cnt] = self._key_ptrs(n, keys, "pkh")
                if nst:
                    hp[2, :nst] = self.store.A_ptrs(n, keys[:nst], st)
                slot.d_ptr.copy_(slot.h_ptr, non_blocking=True)
                if op == "encaps":
                    torch.index_select(P["coins"], 0, rows_d, out=B["coins"][:cnt])
                else:
                    torch.index_select(P["dct"], 0, rows_d, out=B["ct"][:cnt])
                for lo, hi, stored in ((0, nst, True), (nst, cnt, False)):
                    if hi <= lo:
                        continue
                    d0, d1, d2 = slot.d_ptr[0, lo:hi], slot.d_ptr[1, lo:hi], slot.d_ptr[2, lo:hi]
                    if op == "encaps":
                        ctx.encaps_multi(d0, B["coins"][lo:hi], B["ct"][lo:hi], B["K"][lo:hi],
                                         pkh_ptrs=d1, A_ptrs=d2 if stored else None, stream=st)
                    else:
                        ctx.decaps_multi(d0, B["ct"][lo:hi], B["K"][lo:hi],
                                         A_ptrs=d2 if stored else None, stream=st)
                if op == "encaps":
                    P["ct"].index_copy_(0, rows_d, B["ct"][:cnt])
                P["K"].index_copy_(0, rows_d, B["K"][:cnt])
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
        if op != "keygen":
            self.store.used_by(n, {q.key for q in group}, ev)
        slot.event, slot.reqs = ev, group
        self.spans.append((t_start, ev))

    def _take(self, fifo: collections.deque, per_key: collections.Counter, mb: int):
        """The batch to launch from one (operation, n) queue."""
        if fifo[0].op != 0 and not self.cfg.plain:
            key, cnt = per_key.most_common(1)[0]
            if cnt >= self.HOT:
                group, keep = [], collections.deque()
                while fifo:
                    q = fifo.popleft()
                    (group if q.key == key and len(group) < mb else keep).append(q)
                fifo.extend(keep)
                per_key[key] -= len(group)
                return group, True
        group = [fifo.popleft() for _ in range(min(mb, len(fifo)))]
        for q in group:
            per_key[q.key] -= 1
        # one key (a lone request at low load): the plain single-key call
        return group, self.cfg.plain or len({q.key for q in group}) == 1

    def warmup(self):
        """Push one small batch of every kind (KeyGen; single-key and
        multi-key Encaps / Decaps with stored and regenerated A; the tensor
        path) through every slot, so that first-use costs of kernels and
        streams stay out of the measured run.  Results go to scratch rows."""
        for slot in self.slots:
            for n in self.store.params:
                P = self.pool[n]
                reqs = [q for q in self.reqs if q.n == n][:1]
                if not reqs:
                    continue
                base = reqs[0]
                for op in range(3):
                    for single in (True, False):
                        for key in (0, self.cfg.keys_per_n - 1):
                            q = Request(base.rid, op, n, key if op else -1, 0.0)
                            k = min(self.cfg.max_batch, 2 if self.cfg.plain else
                                    (self.HOT if single and op else 2))
                            self._launch(slot, [q] * (1 if self.cfg.plain else k),
                                         single or self.cfg.plain)
                            slot.event.synchronize()
                            slot.event, slot.reqs = None, []
        torch.cuda.synchronize(self.dev)
        self.store.hits = self.store.misses = 0
        self.spans = []
        self.n_single = self.n_multi = self.n_tensor = 0

    def _gpu_busy(self) -> float:
        """Fraction of the span from the first batch's start to the last
        batch's end during which at least one batch was on the device (its
        slot stream between the batch's first and last command)."""
        if not self.spans:
            return 0.0
        ref = self.spans[0][0]
        iv = sorted((ref.elapsed_time(a), ref.elapsed_time(b)) for a, b in self.spans)
        busy, cur_a, cur_b = 0.0, iv[0][0], iv[0][1]
        for a, b in iv[1:]:
            if a > cur_b:
                busy += cur_b - cur_a
                cur_a, cur_b = a, b
            else:
                cur_b = max(cur_b, b)
        busy += cur_b - cur_a
        total = max(b for _, b in iv) - iv[0][0]
        return busy / total if total > 0 else 0.0

    def run(self) -> dict:
        cfg = self.cfg
        mb = 1 if cfg.plain else cfg.max_batch
        fifos: dict = {}
        counts: dict = {}
        nxt, done = 0, 0
        N = len(self.reqs)
        batches = 0
        host_launch = 0.0
        fills0 = self.store.fills
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        while done < N:
            now = time.perf_counter() - t0
            while nxt < N and self.reqs[nxt].t_arr <= now:
                q = self.reqs[nxt]
                k = (q.op, q.n)
                fifos.setdefault(k, collections.deque()).append(q)
                counts.setdefault(k, collections.Counter())[q.key] += 1
                nxt += 1
            for s in self.slots:
                if s.event is not None and s.event.query():
                    tnow = time.perf_counter() - t0
                    for q in s.reqs:
                        q.t_done = tnow
                    done += len(s.reqs)
                    s.event, s.reqs = None, []
            for s in self.slots:
                live = [k for k, f in fifos.items() if f]
                if s.event is not None or not live:
                    continue
                k = min(live, key=lambda k: fifos[k][0].t_arr)  # oldest waiting request
                group, single = self._take(fifos[k], counts[k], mb)
                tl = time.perf_counter()
                self._launch(s, group, single)
                host_launch += time.perf_counter() - tl
                batches += 1
        makespan = max(q.t_done for q in self.reqs) - self.reqs[0].t_arr
        lat = np.array([q.t_done - q.t_arr for q in self.reqs])
        out = {"requests": N, "rate": cfg.rate, "ops_per_s": N / makespan,
               "p50_ms": float(np.percentile(lat, 50) * 1e3),
               "p99_ms": float(np.percentile(lat, 99) * 1e3),
               "batches": batches, "mean_batch": N / max(batches, 1),
               "a_cache_hits": self.store.hits, "a_cache_misses": self.store.misses,
               "a_cache_fills": self.store.fills - fills0, "host_launch_s": host_launch,
               "makespan_s": makespan, "plain": cfg.plain,
               "single_key_batches": self.n_single, "multi_key_batches": self.n_multi,
               "tensor_batches": self.n_tensor, "a_cache_bytes": self.store.used,
               "gpu_busy": self._gpu_busy()}
        by_op = {}
        for i, name in enumerate(OPS):
            li = np.array([q.t_done - q.t_arr for q in self.reqs if q.op == i])
            if len(li):
                by_op[name] = {"count": int(len(li)), "p50_ms": float(np.percentile(li, 50) * 1e3),
                               "p99_ms": float(np.percentile(li, 99) * 1e3)}
        out["by_op"] = by_op
        return out

    # ---- results (for checking) -------------------------------------------
    def result(self, q: Request):
        P = self.pool[q.n]
        row = P["row"][q.rid]
        op = OPS[q.op]
        if op == "keygen":
            return P["pk"][row], P["sk"][row]
        if op == "encaps":
            return P["ct"][row], P["K"][row]
        return P["K"][row], P["dK"][row]


def main():
    """Rate sweep of the served mix against per-request plain launches:
    python -m paper_2606_01211_gb300.serve [--rates 1e3,1e4,...] [--requests N]"""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="1e3,3e3,1e4,3e4,1e5,3e5,1e6")
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--keys-per-n", type=int, default=2500)
    ap.add_argument("--max-batch", type=int, default=512)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--a-budget-gb", type=float, default=None,
                    help="A cache cap (default: none; the cache grows while the live free "
                         "device memory stays above the reserve)")
    ap.add_argument("--no-plain", action="store_true")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    base = ServeConfig(keys_per_n=args.keys_per_n, requests=args.requests,
                       max_batch=args.max_batch, slots=args.slots,
                       a_budget_bytes=None if args.a_budget_gb is None
                       else int(args.a_budget_gb * (1 << 30)))
    store = KeyStore(base, torch.device("cuda", 0))
    for rate in [float(x) for x in args.rates.split(",")]:
        for plain in ([False] if args.no_plain else [False, True]):
            cfg = ServeConfig(**{**base.__dict__, "rate": rate, "plain": plain,
                                 "requests": min(args.requests, max(2000, int(rate * 2)))
                                 if plain else args.requests})
            eng = Engine(cfg, store=store)
            eng.warmup()
            st = eng.run()
            print(json.dumps(st), flush=True)


if __name__ == "__main__":
    main()
