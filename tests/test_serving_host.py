"""Host logic of the continuous-batching server (serving.Server), on the CPU.

The server's scheduling (admission into the open batch of a bucket, the
memory-ledger check, the launch rules: full, a stream idle, max_wait reached,
drain at the end; retirement by completion events; slot strides of the three
batch forms) is plain host code. Here it runs against stand-ins: the CUDA
streams and events of torch are replaced by host clocks (each stream is busy
until the end of the work queued on it; an event fires when its stream's work
has ended), and the library's MulLinRS calls by a stand-in that checks its
arguments (sizes, scratch, key and context, job counts) and writes a
per-slot function of the slot's own input. Each request's result is then
compared with that function of the request's own pooled input, so a request
routed to another slot, bucket or stride fails. The real kernels behind the
same server are tested on the GPU by tests/test_gpu_runtime.py."""
import contextlib
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2109_14704_gb300 import serving  # noqa: E402
from paper_2109_14704_gb300.synth import Rng  # noqa: E402


# ---- stand-ins for CUDA streams and events (host clocks)

class _Stream:
    def __init__(self, device=None):
        self.ready = 0.0                       # host time at which the queued work ends

    def wait_stream(self, other):
        self.ready = max(self.ready, other.ready)


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        now = time.perf_counter()
        self.t = max(now, stream.ready) if stream is not None else now

    def query(self):
        return time.perf_counter() >= self.t

    def synchronize(self):
        time.sleep(max(0.0, self.t - time.perf_counter()))

    def elapsed_time(self, end):
        return (end.t - self.t) * 1e3


def _scratch_need(N, level, count):
    return 8 * count * (level + 1) * N // 4


class _Ctx:
    def __init__(self, N, data, P):
        self.N, self.data_moduli, self.P = int(N), list(data), int(P)

    @property
    def n_data(self):
        return len(self.data_moduli)

    def mrr_scratch_bytes(self, level, count, expand_group=None):
        return _scratch_need(self.N, level, count)

    def mrr_batch_scratch_bytes(self, jobs):
        return sum(_scratch_need(self.N, j[1], j[0]) for j in jobs)


class _Key:
    def __init__(self, ctx, evk):
        assert evk.shape == (ctx.n_data, 2, ctx.n_data + 1, ctx.N)
        self.ctx = ctx


def expected(src, level, N):
    """The stand-in's result for one request: src is the pooled [2 a/b][2][n][N]
    pair; limbs 0..level-1 of 3a + b + level (the rescale drops limb `level`)."""
    a, b = src[0], src[1]
    return (a[:, :level] * 3 + b[:, :level] + level).reshape(-1)


class _He:
    """The library calls the server makes, with argument checks."""
    MAX_BATCH_JOBS = 16

    def __init__(self, cost_s):
        self.cost = cost_s
        self.calls = []                        # (host time, [(N, level, count)], gpu start, gpu end)
        self.default_stream = _Stream()

    @staticmethod
    def chain_primes(N, data_bits, special_bits):
        data = [1000003 + 2 * N + 6 * i for i in range(len(data_bits))]
        return data, 999983

    Context = _Ctx
    RelinKey = _Key

    @staticmethod
    def mul_relin_rescale_multi_scratch_bytes(jobs):
        return sum(_scratch_need(ctx.N, level, count) for count, level, key, ctx in jobs)

    def _run(self, stream, jobs, scratch):
        need = sum(_scratch_need(N, level, count) for N, level, count, _, _, _ in jobs)
        assert scratch.numel() * 8 >= need, "scratch smaller than the batch needs"
        for N, level, count, out, a, b in jobs:
            n = level + 1
            assert a.numel() == count * 2 * n * N and b.numel() == a.numel()
            assert out.numel() == count * 2 * level * N
            A, B = a.view(count, 2, n, N), b.view(count, 2, n, N)
            out.view(count, 2, level, N).copy_(A[:, :, :level] * 3 + B[:, :, :level] + level)
        s = stream if stream is not None else self.default_stream
        now = time.perf_counter()
        start = max(now, s.ready)
        s.ready = start + self.cost
        self.calls.append((now, [(N, level, count) for N, level, count, _, _, _ in jobs], start, s.ready))

    def mul_relin_rescale(self, out, a, b, count, key, ctx, level, scratch, stream=None):
        assert key.ctx is ctx and 1 <= level < ctx.n_data
        self._run(stream, [(ctx.N, level, count, out, a, b)], scratch)

    def mul_relin_rescale_batch(self, jobs, key, ctx, scratch, stream=None):
        assert key.ctx is ctx and 1 <= len(jobs) <= self.MAX_BATCH_JOBS
        self._run(stream, [(ctx.N, level, count, out, a, b) for out, a, b, count, level in jobs], scratch)

    def mul_relin_rescale_multi(self, jobs, scratch, stream=None):
        assert 1 <= len(jobs) <= self.MAX_BATCH_JOBS
        for out, a, b, count, level, key, ctx in jobs:
            assert key.ctx is ctx
        self._run(stream, [(ctx.N, level, count, out, a, b) for out, a, b, count, level, key, ctx in jobs], scratch)


@pytest.fixture
def fake(monkeypatch):
    def make(cost_s):
        he = _He(cost_s)
        monkeypatch.setattr(serving, "he", he)
        monkeypatch.setattr(torch.cuda, "Stream", _Stream)
        monkeypatch.setattr(torch.cuda, "Event", _Event)
        monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
        monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
        return he
    return make


def _pool(degrees, min_level, max_level, per_bucket, seed):
    r = Rng(seed)
    pool = {}
    for N in degrees:
        for lvl in range(min_level, max_level + 1):
            qs = [1000003 + 6 * i for i in range(lvl + 1)]
            pairs = np.stack([np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
                                        for _ in range(2)]) for _ in range(per_bucket)])
            pool[(N, lvl)] = torch.from_numpy(pairs.astype(np.int64))
    return pool


def _server(degrees=(16, 32), min_level=1, max_level=4, per_bucket=3, **kw):
    args = dict(degrees=degrees, min_level=min_level, max_level=max_level, slots=4, streams=2, max_wait_s=0.001,
                seed=3, device=torch.device("cpu"),
                pool=_pool(degrees, min_level, max_level, per_bucket, 4))
    args.update(kw)
    return serving.Server(**args)


_MODES = {"per_level": {}, "mixed_levels": {"mixed_levels": True}, "mixed_degrees": {"mixed_degrees": True}}


@pytest.mark.parametrize("mode", list(_MODES))
def test_every_request_gets_its_own_result(fake, mode):
    he = fake(0.0004)
    srv = _server(**_MODES[mode])
    reqs = srv.make_requests(300, rate=20000.0, seed=6)
    stats = srv.run(reqs, keep_ids=range(300))
    assert stats["requests"] == 300 and len(srv.completed) == 300
    assert sorted(r.rid for r in srv.completed) == list(range(300))
    for r in reqs:
        src = srv.pool[(r.N, r.level)][r.src]
        assert torch.equal(srv.keep[r.rid], expected(src, r.level, r.N)), r.rid
        assert r.done >= r.arrival
    # batches: at most `slots` requests; one (degree, level) per call, one
    # degree per mixed-level call; batching engaged at this rate
    sizes = [sum(c for _, _, c in jobs) for _, jobs, _, _ in he.calls]
    assert sum(sizes) == 300 and max(sizes) <= srv.slots
    assert len(he.calls) == stats["batches"] < 300
    for _, jobs, _, _ in he.calls:
        if mode == "per_level":
            assert len(jobs) == 1
        elif mode == "mixed_levels":
            assert len({N for N, _, _ in jobs}) == 1
    if mode != "per_level":
        assert any(len({lv for _, lv, _ in jobs}) > 1 for _, jobs, _, _ in he.calls)
    if mode == "mixed_degrees":
        assert any(len({N for N, _, _ in jobs}) > 1 for _, jobs, _, _ in he.calls)
    # every buffer went back to the cache; the ledger stayed in budget
    assert srv.cache.in_use == 0 and not srv.inflight and not srv.open
    assert srv.peak_ledger <= srv.budget


@pytest.mark.parametrize("mode", list(_MODES))
def test_alone_equals_in_the_mix(fake, mode):
    fake(0.0002)
    srv = _server(**_MODES[mode])
    reqs = srv.make_requests(60, rate=20000.0, seed=7)
    srv.run(reqs, keep_ids=[0, 17, 59])
    for rid in (0, 17, 59):
        assert torch.equal(srv.keep[rid], srv.serve_alone(reqs[rid])), rid


def _reqs(spec):
    """spec: (arrival_s, N, level) per request; first pooled pair."""
    return [serving.Request(i, t, N, lvl, 0) for i, (t, N, lvl) in enumerate(spec)]


def test_a_partial_batch_waits_max_wait_while_every_stream_is_busy(fake):
    """r0 finds the only stream idle and goes alone; r1 and r2 arrive while it
    runs and wait in the open batch until the oldest of them has waited
    max_wait, long before the stream frees; r3 (much later) keeps the queue
    non-empty meanwhile."""
    he = fake(0.050)
    srv = _server(degrees=(16,), slots=8, streams=1, max_wait_s=0.002)
    srv.run(_reqs([(0.0, 16, 2), (0.005, 16, 2), (0.0051, 16, 2), (0.2, 16, 2)]))
    sizes = [sum(c for _, _, c in jobs) for _, jobs, _, _ in he.calls]
    assert sizes == [1, 2, 1]
    t_launch = he.calls[1][0] - srv.t0_host
    assert 0.005 + 0.002 <= t_launch < 0.045


def test_a_full_batch_launches_at_once(fake):
    he = fake(0.050)
    srv = _server(degrees=(16,), slots=2, streams=1, max_wait_s=1.0)
    srv.run(_reqs([(0.0, 16, 2), (0.005, 16, 2), (0.0055, 16, 2), (0.2, 16, 2)]))
    sizes = [sum(c for _, _, c in jobs) for _, jobs, _, _ in he.calls]
    assert sizes == [1, 2, 1]
    assert he.calls[1][0] - srv.t0_host < 0.045       # full: no wait for the stream or max_wait


def test_the_last_requests_drain_without_waiting(fake):
    he = fake(0.030)
    srv = _server(degrees=(16,), slots=8, streams=1, max_wait_s=1.0)
    srv.run(_reqs([(0.0, 16, 2), (0.002, 16, 2), (0.0021, 16, 2)]))
    sizes = [sum(c for _, _, c in jobs) for _, jobs, _, _ in he.calls]
    assert sizes == [1, 2]
    assert he.calls[1][0] - srv.t0_host < 0.025       # not held for max_wait


def test_buckets_never_mix_in_per_level_batches(fake):
    he = fake(0.050)
    srv = _server(degrees=(16, 32), slots=8, streams=1, max_wait_s=0.002)
    spec = [(0.0, 16, 2), (0.003, 16, 2), (0.0031, 32, 2), (0.0032, 16, 3), (0.0033, 16, 2), (0.2, 16, 2)]
    srv.run(_reqs(spec), keep_ids=range(len(spec)))
    got = sorted(tuple(jobs) for _, jobs, _, _ in he.calls)
    assert got == sorted([((16, 2, 1),), ((16, 2, 2),), ((32, 2, 1),), ((16, 3, 1),), ((16, 2, 1),)])
    for i, (t, N, lvl) in enumerate(spec):
        assert torch.equal(srv.keep[i], expected(srv.pool[(N, lvl)][0], lvl, N)), i


def test_admission_waits_for_memory(fake):
    """A budget with room for one batch: the next batch is opened only after
    the previous one retired, so the batches never overlap on the device,
    and every request is still served."""
    he = fake(0.002)
    srv = _server(degrees=(32,), min_level=3, max_level=3, slots=2, streams=2, max_wait_s=0.0005)
    one = sum(srv.cache._capacity(w) for w in srv._batch_words(32, 3, 2)) * 8
    srv.budget = srv.static_bytes + one + one // 2
    reqs = srv.make_requests(40, rate=20000.0, seed=8)
    stats = srv.run(reqs, keep_ids=range(40))
    assert len(srv.completed) == 40 and srv.peak_ledger <= srv.budget
    spans = sorted((start, end) for _, _, start, end in he.calls)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0, "two batches held memory at once"
    for r in reqs:
        assert torch.equal(srv.keep[r.rid], expected(srv.pool[(32, 3)][r.src], 3, 32)), r.rid
    assert stats["cache_misses"] == 4               # one set of four buffers, reused by every batch


def test_no_room_for_a_single_batch_is_an_error_not_a_hang(fake):
    """With nothing in flight or open, no memory can come free: a batch that
    does not fit the budget by itself is refused instead of waited for."""
    fake(0.001)
    srv = _server(degrees=(32,), min_level=3, max_level=3, slots=2)
    srv.budget = srv.static_bytes + 8                  # nothing fits
    with pytest.raises(MemoryError, match="budget"):
        srv.run(_reqs([(0.0, 32, 3)]))
    assert srv.cache.reserved == 0
