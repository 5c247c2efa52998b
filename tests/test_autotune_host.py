"""Host logic of the autotuner (autotune.tune_uniform, tune_mul_relin_rescale),
on the CPU: the library's shape and transform calls are replaced by
stand-ins that keep a simulated device clock (each call advances it by the
time scripted for the shape in force) and CUDA events that read that clock.
Checked: every built shape is tried in both launch forms, a candidate whose
forward output differs from the default shape's or whose inverse does not
restore the input is never chosen however fast it is, each direction gets
its own fastest shape, ties go to the earlier candidate, the default shape
is restored after tuning (also when a call fails), the cache is used and
`force` re-tunes, and the chosen shapes are applied per direction. The real
shapes are tuned and checked against the oracle on the GPU by
tests/test_gpu_runtime.py and tests/test_gpu_ntt.py."""
import pytest

torch = pytest.importorskip("torch")

from paper_2109_14704_gb300 import autotune  # noqa: E402


class _Clock:
    t = 0.0


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = _Clock.t

    def synchronize(self):
        pass

    def elapsed_time(self, end):
        return end.t - self.t


class _He:
    FORWARD, INVERSE, BOTH = 1, 2, 0

    def __init__(self, shapes, ms, broken=(), fail=None):
        self.shapes = list(shapes)             # (log_block, log_thread_words, ctas_per_sm), default first
        self.ms = ms                           # (shape4, "fwd"|"inv") -> ms per call
        self.broken = set(broken)              # (shape4, "fwd"|"inv"): wrong results
        self.fail = fail                       # shape4 whose forward raises
        self.cur = {self.FORWARD: None, self.INVERSE: None}
        self.set_calls = []

    def ntt_shapes(self, N):
        return list(self.shapes)

    def ntt_set_shape(self, N, log_block=0, log_thread_words=0, persistent=0, direction=0, ctas_per_sm=0):
        shape = None if (log_block, log_thread_words, persistent, ctas_per_sm) == (0, 0, 0, 0) else \
            (log_block, log_thread_words, persistent, ctas_per_sm)
        self.set_calls.append((direction, shape))
        for d in ((self.FORWARD, self.INVERSE) if direction == self.BOTH else (direction,)):
            self.cur[d] = shape

    def _shape(self, d):
        lb, le, occ = self.shapes[0]
        return self.cur[d] or (lb, le, 0, occ)

    @staticmethod
    def primes_generate(bits, two_n, count):
        return [(1 << bits) - 1 - 2 * two_n * i for i in range(count)]

    class NttTables:
        def __init__(self, N, qs):
            self.N, self.moduli = N, list(qs)

    def ntt_fwd(self, d, N, limbs, count, tables):
        s = self._shape(self.FORWARD)
        if s == self.fail:
            raise RuntimeError("launch failed")
        d.add_(8 if (s, "fwd") in self.broken else 7)
        _Clock.t += self.ms.get((s, "fwd"), 10.0)

    def ntt_inv(self, d, N, limbs, count, tables):
        s = self._shape(self.INVERSE)
        d.sub_(6 if (s, "inv") in self.broken else 7)
        _Clock.t += self.ms.get((s, "inv"), 10.0)


@pytest.fixture
def fake(monkeypatch):
    def make(**kw):
        he = _He(**kw)
        monkeypatch.setattr(autotune, "he", he)
        monkeypatch.setattr(autotune, "_device_key", lambda: "test-device")
        monkeypatch.setattr(torch.cuda, "Event", _Event)
        monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
        monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
        empty = torch.empty
        monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: empty(*a, **k))
        return he
    return make


SHAPES = [(12, 4, 0), (12, 3, 0), (11, 4, 0)]


def _s(i, pers=0):
    lb, le, occ = SHAPES[i]
    return (lb, le, pers, occ)


def test_every_shape_in_both_launch_forms_and_each_direction_its_fastest(fake, tmp_path):
    ms = {(_s(1), "fwd"): 3.0, (_s(2, 1), "inv"): 2.0, (_s(0), "fwd"): 5.0, (_s(0), "inv"): 5.0}
    he = fake(shapes=SHAPES, ms=ms)
    res = autotune.tune_uniform(1024, 2, 3, reps=3, warmup=1, cache_path=str(tmp_path / "c.json"))
    assert [tuple(c["shape"]) for c in res["candidates"]] == [_s(i, p) for p in (0, 1) for i in range(3)]
    assert all(c["ok"] for c in res["candidates"])
    assert tuple(res["fwd"]) == _s(1) and tuple(res["inv"]) == _s(2, 1)
    assert res["ms_fwd"] == 3.0 and res["ms_inv"] == 2.0 and res["default_ms_fwd_inv"] == 10.0
    # applied per direction, after the default was restored
    assert he.set_calls[-3] == (he.BOTH, None)
    assert he.set_calls[-2:] == [(he.FORWARD, _s(1)), (he.INVERSE, _s(2, 1))]


def test_a_wrong_candidate_is_never_chosen(fake, tmp_path):
    ms = {(_s(2), "fwd"): 0.1, (_s(1), "inv"): 0.1, (_s(0, 1), "fwd"): 4.0, (_s(0), "inv"): 4.0}
    fake(shapes=SHAPES, ms=ms, broken={(_s(2), "fwd"), (_s(1), "inv")})
    res = autotune.tune_uniform(1024, 2, 3, reps=3, warmup=1, cache_path=str(tmp_path / "c.json"))
    bad = {tuple(c["shape"]) for c in res["candidates"] if not c["ok"]}
    assert bad == {_s(2), _s(1)}
    assert all("ms_fwd" not in c for c in res["candidates"] if not c["ok"])   # never timed
    assert tuple(res["fwd"]) == _s(0, 1) and tuple(res["inv"]) == _s(0)


def test_ties_go_to_the_earlier_candidate(fake, tmp_path):
    fake(shapes=SHAPES, ms={})                   # every shape 10 ms
    res = autotune.tune_uniform(1024, 2, 3, reps=3, warmup=1, cache_path=None)
    assert tuple(res["fwd"]) == _s(0) and tuple(res["inv"]) == _s(0)


def test_no_passing_shape_is_an_error(fake):
    fake(shapes=SHAPES[:1], ms={}, broken={(_s(0), "inv"), (_s(0, 1), "inv")})
    with pytest.raises(RuntimeError, match="passed its check"):
        autotune.tune_uniform(1024, 2, 3, reps=2, warmup=1, cache_path=None)


def test_default_restored_when_a_candidate_fails(fake):
    he = fake(shapes=SHAPES, ms={}, fail=_s(1))
    with pytest.raises(RuntimeError, match="launch failed"):
        autotune.tune_uniform(1024, 2, 3, reps=2, warmup=1, cache_path=None)
    assert he.set_calls[-1] == (he.BOTH, None) and he.cur == {he.FORWARD: None, he.INVERSE: None}


def test_cached_result_is_applied_without_timing_and_force_retunes(fake, tmp_path):
    path = str(tmp_path / "c.json")
    fake(shapes=SHAPES, ms={(_s(1), "fwd"): 1.0, (_s(1), "inv"): 1.0})
    first = autotune.tune_uniform(1024, 2, 3, reps=2, warmup=1, cache_path=path)
    # a second tuner whose timings differ: the cache answers, nothing runs
    he2 = fake(shapes=SHAPES, ms={(_s(2), "fwd"): 0.5, (_s(2), "inv"): 0.5})
    t0 = _Clock.t
    again = autotune.tune_uniform(1024, 2, 3, reps=2, warmup=1, cache_path=path)
    assert _Clock.t == t0 and again["fwd"] == first["fwd"] == list(_s(1))
    assert he2.set_calls == [(he2.FORWARD, _s(1)), (he2.INVERSE, _s(1))]
    # another batch shape is another cache entry; force re-tunes this one
    assert tuple(autotune.tune_uniform(1024, 2, 4, reps=2, warmup=1, cache_path=path)["fwd"]) == _s(2)
    assert tuple(autotune.tune_uniform(1024, 2, 3, reps=2, warmup=1, cache_path=path, force=True)["fwd"]) == _s(2)
    assert len(autotune._load_cache(path)) == 2


class _Ctx:
    N = 64
    data_moduli = [97, 193, 257]

    def __init__(self, broken=None, ms=None):
        self.shape, self.set_calls = 0, []
        self.broken, self.ms = broken, ms or {}

    def set_eval_shape(self, le):
        self.shape = le
        self.set_calls.append(le)

    def mrr_scratch_bytes(self, level, count):
        return 8 * count


def test_mul_relin_rescale_radix_needs_the_default_output(fake, monkeypatch):
    fake(shapes=SHAPES, ms={})
    for broken, ms, want in ((None, {4: 2.0, 3: 1.0}, 3), (3, {4: 2.0, 3: 1.0}, 4), (None, {4: 1.0, 3: 1.0}, 4)):
        ctx = _Ctx(broken, ms)

        def mrr(out, a, b, count, key, c, level, scratch, stream=None):
            out.copy_((a[:, :, :level] + b[:, :, :level]) + (1 if c.shape == c.broken else 0))
            _Clock.t += c.ms.get(c.shape, 5.0)
        monkeypatch.setattr(autotune.he, "mul_relin_rescale", mrr, raising=False)
        res = autotune.tune_mul_relin_rescale(ctx, None, 2, 3, reps=2, warmup=1)
        assert res["log_thread_words"] == want, (broken, ms)
        assert [c["ok"] for c in res["candidates"]] == [broken != 4, broken != 3]
        assert ctx.set_calls[0] == 0 and ctx.set_calls[-1] == want      # default first, the choice applied
