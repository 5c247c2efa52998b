"""Continuous-batching request loop for mul-relin-rescale (MulLinRS) jobs.

The paper's client/server flow (Sec. III): the host encrypts, ships
ciphertexts and static data (keys) to the GPU once, the GPU evaluates
asynchronously and the host synchronises only to read results back; device
buffers come from a memory cache that reuses any free buffer large enough
(Sec. III-C, "memory cache"). This module turns that into a server:

* Requests (N, level, input pair) arrive by an open-loop Poisson process.
* Relinearization keys of every degree stay resident on the device.
* A request is admitted into the open batch of its (N, level) bucket as soon
  as the batch has a free slot and the device-memory ledger (keys + tables +
  every buffer the memory cache holds, against an HBM budget; free cached
  buffers are evicted to make room) can hold the batch; its
  input ciphertexts are copied from pinned host memory straight into the
  batch slot.
* A bucket's open batch is launched (one he_mul_relin_rescale call over all
  its slots) when it is full, when a stream is idle, or when its oldest
  request has waited max_wait_s; meanwhile new arrivals fill the next open
  batch (continuous batching), and batches in flight on several streams
  overlap on the device.
* With mixed_levels, the buckets are the degrees alone: a batch takes
  requests of any level (each slot sized for the highest level) and runs as
  one he_mul_relin_rescale_batch call, one launch per pipeline stage for the
  whole mix (each request one job). With mixed_degrees, one bucket takes
  every degree and level (slots sized for the largest of both) and runs as
  one he_mul_relin_rescale_multi call: jobs of different degrees share one
  launch per pipeline stage.
* Completion is timed with CUDA events; latency = completion - arrival on
  one clock (events are anchored to the host clock at start). Buffers go
  back to the memory cache when the batch's completion event has fired.
"""
from __future__ import annotations

import bisect
import collections
import gc
import math
import statistics
import time
from dataclasses import dataclass, field

import numpy as np

from . import he
from .synth import Rng


class DeviceMemoryCache:
    """Device buffer pool: allocate reuses the smallest free buffer with
    capacity at least the request, else allocates; free returns a buffer to
    the pool. `reserved` (bytes held, free or in use) is what the admission
    ledger counts; free buffers can be evicted to make room.

    Free buffers stay sorted by capacity, so a pick is a binary search (the
    serving loop runs on one host thread and may hold thousands of buffers).
    With size_classes, new buffers are rounded up to the next of the sizes
    2^(k/4) words (at most 19 % slack), so that a buffer freed by one
    (N, level) bucket serves its neighbours instead of each bucket growing
    its own."""

    def __init__(self, device, size_classes: bool = False):
        import torch
        self.torch = torch
        self.device = device
        self.size_classes = size_classes
        self._free: list = []              # sorted (capacity_words, seq, tensor)
        self._seq = 0
        self.reserved = 0                  # bytes held by the cache (free + in use)
        self.in_use = 0
        self.hits = 0
        self.misses = 0
        self.evicted = 0

    @property
    def free_list(self):
        return [(cap, t) for cap, _, t in self._free]

    def _capacity(self, words: int) -> int:
        if not self.size_classes or words <= 256:
            return words
        k = math.ceil(4 * math.log2(words))
        while 2 ** ((k - 1) / 4) >= words:     # guard the float rounding
            k -= 1
        return int(math.ceil(2 ** (k / 4) / 256)) * 256

    def _pick(self, words, taken):
        """Index into the free list of the smallest buffer of >= words
        words that is not in `taken`, or None."""
        i = bisect.bisect_left(self._free, (words, -1))
        while i < len(self._free) and i in taken:
            i += 1
        return i if i < len(self._free) else None

    def growth(self, words_list) -> int:
        """Bytes of new memory that allocating all of words_list would add."""
        taken, grow = set(), 0
        for w in words_list:
            i = self._pick(w, taken)
            if i is None:
                grow += self._capacity(w) * 8
            else:
                taken.add(i)
        return grow

    def allocate_within(self, words_list, limit_bytes: int, base_bytes: int = 0):
        """Allocate every request of words_list so that base_bytes + reserved
        stays within limit_bytes, evicting free buffers (largest first) when
        that makes room; None (and nothing allocated) if it cannot."""
        while base_bytes + self.reserved + self.growth(words_list) > limit_bytes:
            taken = set()
            for w in words_list:
                i = self._pick(w, taken)
                if i is not None:
                    taken.add(i)
            j = len(self._free) - 1
            while j >= 0 and j in taken:
                j -= 1
            if j < 0:
                return None
            cap, _, _ = self._free.pop(j)
            self.reserved -= cap * 8
            self.evicted += 1
        return [self.allocate(w) for w in words_list]

    def allocate(self, words: int):
        best = self._pick(words, set())
        if best is not None:
            cap, _, t = self._free.pop(best)
            self.hits += 1
        else:
            cap = self._capacity(words)
            t = self.torch.empty(cap, dtype=self.torch.int64, device=self.device)
            self.reserved += cap * 8
            self.misses += 1
        self.in_use += cap * 8
        return cap, t

    def free(self, cap: int, t):
        self.in_use -= cap * 8
        self._seq += 1
        bisect.insort(self._free, (cap, self._seq, t))


@dataclass
class Request:
    rid: int
    arrival: float
    N: int
    level: int
    src: int                               # index into the host input pool
    done: float = -1.0
    batch: "Batch | None" = None
    slot: int = -1


@dataclass
class Batch:
    key: tuple
    cap: int
    bufs: list = field(default_factory=list)   # (capacity, tensor) for a, b, out, scratch
    reqs: list = field(default_factory=list)
    opened: float = 0.0
    stream: object = None
    done_event: object = None
    launched: bool = False


class Server:
    """MulLinRS server over degrees `degrees` and levels [min_level, max_level]."""

    def __init__(self, degrees=(8192, 16384, 32768), min_level=2, max_level=16, budget_bytes=64 << 30,
                 slots=16, streams=4, max_wait_s=0.002, pool_per_bucket=2, seed=5, device=None, expand_group=4,
                 prewarm_batches=0, mixed_levels=False, mixed_degrees=False, pool=None):
        import torch
        self.torch = torch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.degrees = list(degrees)
        self.min_level, self.max_level = min_level, max_level
        self.budget = budget_bytes
        self.slots = slots
        self.max_wait = max_wait_s
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.busy = {i: None for i in range(streams)}
        self.cache = DeviceMemoryCache(self.device, size_classes=True)
        # key-switching mod-up expanded in groups of at most this many
        # ciphertexts (bounds a batch's scratch; 0 = the fused minimum)
        self.expand_group = expand_group
        # mixed_levels: one batch per degree, any level; mixed_degrees: one
        # batch for every degree and level (he_mul_relin_rescale_multi)
        self.mixed_deg = mixed_degrees
        self.mixed = mixed_levels or mixed_degrees
        if self.mixed and slots > he.MAX_BATCH_JOBS:
            raise ValueError(f"mixed batches take at most {he.MAX_BATCH_JOBS} slots")
        self.rng = Rng(seed)
        self.ctx, self.key, self.moduli = {}, {}, {}
        self.static_bytes = 0
        n_data = max_level + 1
        for N in self.degrees:
            data, P = he.chain_primes(N, [60] + [50] * (n_data - 1), 60)
            self.moduli[N] = data
            self.ctx[N] = he.Context(N, data, P)
            evk = np.stack([np.stack([self.rng.uniform_limbs(data + [P], N) for _ in range(2)])
                            for _ in range(n_data)])
            self.key[N] = he.RelinKey(self.ctx[N], evk)
            # resident: key words with Shoup quotients, twiddles of n_data+1 primes, constants
            self.static_bytes += evk.size * 16 + (n_data + 1) * N * 32
        # Client-side input pool: pinned host ciphertext pairs per (N, level)
        # (or another server's pool over the same degrees and levels).
        self.pool = pool if pool is not None else {}
        for N in ([] if pool is not None else self.degrees):
            for lvl in range(min_level, max_level + 1):
                qs = self.moduli[N][:lvl + 1]
                pairs = np.stack([np.stack([np.stack([self.rng.uniform_limbs(qs, N) for _ in range(2)])
                                            for _ in range(2)]) for _ in range(pool_per_bucket)])
                self.pool[(N, lvl)] = torch.from_numpy(pairs.view(np.int64)).pin_memory()  # [P][2 a/b][2][n][N]
        self.open = {}
        self.inflight: list[Batch] = []
        self.waiting: collections.deque = collections.deque()
        self.completed: list[Request] = []
        self.keep: dict = {}                   # rid -> result copy (host) for requests to check
        self.peak_ledger = 0
        self.batches_launched = 0
        if prewarm_batches:
            self.prewarm(prewarm_batches)

    def prewarm(self, batches: int):
        """Reserve the memory pool up front, as a server does at start-up:
        `batches` buffer sets of the largest bucket (any smaller batch can
        reuse them), allocated and returned to the cache, so that requests
        seldom wait for the device allocator."""
        N, lvl = max(self.degrees), self.max_level
        words = self._batch_words(N, lvl, self.slots)   # also the mixed form's size
        sets = []
        for _ in range(batches):
            got = self.cache.allocate_within(words, self.budget, self.static_bytes)
            if got is None:
                break
            sets.append(got)
        for got in sets:
            for cap, t in got:
                self.cache.free(cap, t)
        self.peak_ledger = max(self.peak_ledger, self.ledger())

    # ---- ledger
    def ledger(self) -> int:
        return self.static_bytes + self.cache.reserved

    def _batch_words(self, N, lvl, cap):
        n = lvl + 1
        ct_in = 2 * n * N
        if self.mixed_deg:   # slots sized for the largest degree and level
            scratch = he.mul_relin_rescale_multi_scratch_bytes([(1, lvl, self.key[N], self.ctx[N])] * cap) // 8
        elif self.mixed:     # slots sized for the highest level
            scratch = self.ctx[N].mrr_batch_scratch_bytes([(1, lvl)] * cap) // 8
        else:
            scratch = self.ctx[N].mrr_scratch_bytes(lvl, cap, self.expand_group) // 8
        return [cap * ct_in, cap * ct_in, cap * 2 * lvl * N, scratch]

    def _slot_words(self, N, lvl):
        """Input and output words of one slot of a batch (its stride)."""
        if self.mixed_deg:
            N = max(self.degrees)
        if self.mixed:
            lvl = self.max_level
        return 2 * (lvl + 1) * N, 2 * lvl * N

    def _open_batch(self, key, now):
        N, lvl = key
        if self.mixed_deg:
            N = max(self.degrees)
        words = self._batch_words(N, self.max_level if self.mixed else lvl, self.slots)
        bufs = self.cache.allocate_within(words, self.budget, self.static_bytes)
        if bufs is None:
            return None
        b = Batch(key=key, cap=self.slots, opened=now)
        b.bufs = bufs
        self.open[key] = b
        self.peak_ledger = max(self.peak_ledger, self.ledger())
        return b

    # ---- request flow
    def _admit(self, req: Request, now) -> bool:
        key = (None if self.mixed_deg else req.N, None if self.mixed else req.level)
        b = self.open.get(key)
        if b is None:
            b = self._open_batch(key, now)
            if b is None:
                return False
        slot = len(b.reqs)
        per = 2 * (req.level + 1) * req.N
        stride = self._slot_words(req.N, req.level)[0]
        src = self.pool[(req.N, req.level)][req.src]
        a_t, b_t = b.bufs[0][1], b.bufs[1][1]
        # upload of the request's two ciphertexts into the batch slot
        with self.torch.cuda.stream(self.streams[0]):
            a_t[slot * stride:slot * stride + per].copy_(src[0].reshape(-1), non_blocking=True)
            b_t[slot * stride:slot * stride + per].copy_(src[1].reshape(-1), non_blocking=True)
        req.batch, req.slot = b, slot
        b.reqs.append(req)
        if len(b.reqs) == b.cap:
            self._launch(b)
        return True

    def _free_stream(self):
        for i, bt in self.busy.items():
            if bt is None:
                return i
        return None

    def _launch(self, b: Batch, stream_index=None):
        torch = self.torch
        if stream_index is None:
            stream_index = self._free_stream()
            if stream_index is None:
                stream_index = min(self.busy, key=lambda i: self.busy[i].opened if self.busy[i] else 0)
        s = self.streams[stream_index]
        s.wait_stream(self.streams[0])          # the uploads
        N, lvl = b.key
        count = len(b.reqs)
        scratch = b.bufs[3][1]
        if self.mixed_deg:
            si, so = self._slot_words(None, None)
            jobs = []
            for r in b.reqs:
                pi, po = 2 * (r.level + 1) * r.N, 2 * r.level * r.N
                jobs.append((b.bufs[2][1][r.slot * so:r.slot * so + po], b.bufs[0][1][r.slot * si:r.slot * si + pi],
                             b.bufs[1][1][r.slot * si:r.slot * si + pi], 1, r.level, self.key[r.N], self.ctx[r.N]))
            he.mul_relin_rescale_multi(jobs, scratch, stream=s)
        elif self.mixed:
            si, so = self._slot_words(N, None)
            jobs = []
            for r in b.reqs:
                pi, po = 2 * (r.level + 1) * N, 2 * r.level * N
                jobs.append((b.bufs[2][1][r.slot * so:r.slot * so + po], b.bufs[0][1][r.slot * si:r.slot * si + pi],
                             b.bufs[1][1][r.slot * si:r.slot * si + pi], 1, r.level))
            he.mul_relin_rescale_batch(jobs, self.key[N], self.ctx[N], scratch, stream=s)
        else:
            n = lvl + 1
            per_in, per_out = 2 * n * N, 2 * lvl * N
            a = b.bufs[0][1][:count * per_in]
            bb = b.bufs[1][1][:count * per_in]
            out = b.bufs[2][1][:count * per_out]
            he.mul_relin_rescale(out, a, bb, count, self.key[N], self.ctx[N], lvl, scratch, stream=s)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(s)
        b.done_event, b.stream, b.launched = ev, s, True
        self.busy[stream_index] = b
        b.stream_index = stream_index
        self.open.pop(b.key, None)
        self.inflight.append(b)
        self.batches_launched += 1

    def _retire(self):
        still = []
        for b in self.inflight:
            if b.done_event.query():
                t = self.anchor.elapsed_time(b.done_event) / 1e3     # seconds since start
                for r in b.reqs:
                    r.done = t
                    self.completed.append(r)
                    if r.rid in self.keep:
                        so = self._slot_words(r.N, r.level)[1]
                        self.keep[r.rid] = b.bufs[2][1][r.slot * so:r.slot * so + 2 * r.level * r.N].cpu().clone()
                for cap, t_ in b.bufs:
                    self.cache.free(cap, t_)
                if self.busy.get(b.stream_index) is b:
                    self.busy[b.stream_index] = None
            else:
                still.append(b)
        self.inflight = still

    def make_requests(self, n_requests: int, rate: float, seed: int = 5) -> list[Request]:
        r = Rng(seed, stream=1)
        gaps = r.exponential(n_requests, rate)
        arrivals = np.cumsum(gaps)
        degs = r.choice(self.degrees, n_requests)
        lvls = r.choice(list(range(self.min_level, self.max_level + 1)), n_requests)
        srcs = r.choice(list(range(self.pool[(self.degrees[0], self.min_level)].shape[0])), n_requests)
        return [Request(i, float(arrivals[i]), int(degs[i]), int(lvls[i]), int(srcs[i])) for i in range(n_requests)]

    def run(self, requests: list[Request], keep_ids=()) -> dict:
        """Serve `requests` (arrival times in seconds from start) in real time."""
        torch = self.torch
        self.keep = {rid: None for rid in keep_ids}
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
        # no collector pauses inside the serving loop (it runs on one host
        # thread; a full collection of a large process takes milliseconds)
        gc.collect()
        gc_was_enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(pending, torch)
        finally:
            if gc_was_enabled:
                gc.enable()

    def _run(self, pending, torch) -> dict:
        torch.cuda.synchronize()
        self.anchor = torch.cuda.Event(enable_timing=True)
        self.anchor.record(self.streams[0])
        self.anchor.synchronize()
        self.t0_host = time.perf_counter()
        total = len(pending)
        while len(self.completed) < total:
            now = time.perf_counter() - self.t0_host
            while pending and pending[0].arrival <= now:
                self.waiting.append(pending.popleft())
            while self.waiting:
                if not self._admit(self.waiting[0], now):
                    if not self.inflight and not self.open:
                        # nothing holds memory that could be freed: this
                        # request's batch alone exceeds the budget
                        req = self.waiting[0]
                        raise MemoryError(f"a batch of (N={req.N}, level={req.level}) needs more than the "
                                          f"{self.budget} bytes budgeted ({self.static_bytes} held by keys "
                                          f"and tables)")
                    break
                self.waiting.popleft()
            for key, b in list(self.open.items()):
                if b.reqs and (self._free_stream() is not None or now - b.reqs[0].arrival >= self.max_wait):
                    self._launch(b)
            self._retire()
            if not pending and not self.waiting:
                for b in list(self.open.values()):
                    if b.reqs:
                        self._launch(b)
            if pending and not self.inflight and not self.waiting:
                # idle: sleep only while the next arrival is comfortably
                # far, and wake 0.2 ms early (a sleep may overrun by a
                # fraction of a millisecond, which would add to the latency
                # of every request arriving meanwhile); poll otherwise
                gap = pending[0].arrival - now
                if gap > 0.0003:
                    time.sleep(min(gap - 0.0002, 0.0005))
        torch.cuda.synchronize()
        lat = [(r.done - r.arrival) * 1e3 for r in self.completed]
        span = max(r.done for r in self.completed) - min(r.arrival for r in self.completed)
        return {
            "requests": total,
            "throughput_per_s": total / span if span > 0 else float("nan"),
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": statistics.mean(lat),
            "batches": self.batches_launched,
            "mean_batch": total / max(1, self.batches_launched),
            "peak_ledger_gb": self.peak_ledger / 2 ** 30,
            "budget_gb": self.budget / 2 ** 30,
            "cache_hits": self.cache.hits, "cache_misses": self.cache.misses, "cache_evictions": self.cache.evicted,
        }

    def serve_alone(self, req: Request):
        """The result of one request run by itself (a batch of one)."""
        torch = self.torch
        N, lvl = req.N, req.level
        src = self.pool[(N, lvl)][req.src].to(self.device)
        out = torch.empty(2 * lvl * N, dtype=torch.int64, device=self.device)
        scratch = torch.empty(self.ctx[N].mrr_scratch_bytes(lvl, 1, self.expand_group) // 8, dtype=torch.int64,
                              device=self.device)
        he.mul_relin_rescale(out, src[0].contiguous(), src[1].contiguous(), 1, self.key[N], self.ctx[N], lvl, scratch)
        torch.cuda.synchronize()
        return out.cpu()
