"""GPU tests of the batching runtime: the autotuner (every candidate checked,
choice cached and applied) and the continuous-batching MulLinRS server
(results bit-identical alone and in the mix, admission within the memory
budget, batching under load)."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import autotune, he, serving
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, host  # noqa: E402


def test_autotune_uniform(tmp_path):
    N, limbs, count = 16384, 4, 24
    cache = str(tmp_path / "tune.json")
    res = autotune.tune_uniform(N, limbs, count, reps=3, warmup=1, cache_path=cache)
    shapes = he.ntt_shapes(N)
    for d in ("fwd", "inv"):
        lb, le, pers, occ = res[d]
        assert (lb, le, occ) in shapes and pers in (0, 1)
    assert all(c["ok"] for c in res["candidates"]) and len(res["candidates"]) == 2 * len(shapes)
    assert res["ms_fwd"] == min(c["ms_fwd"] for c in res["candidates"])
    assert res["ms_inv"] == min(c["ms_inv"] for c in res["candidates"])
    again = autotune.tune_uniform(N, limbs, count, cache_path=cache)   # from the cache
    assert again["fwd"] == res["fwd"] and again["inv"] == res["inv"]
    # the applied shape still computes the oracle's transform
    qs = autotune.default_moduli(N, limbs)
    tables = he.NttTables(N, qs)
    x = Rng(5).uniform_limbs(qs, N)
    d = dev(x)
    he.ntt_fwd(d, N, limbs, 1, tables)
    assert np.array_equal(host(d), oracle.ntt_fwd(x, qs))
    he.ntt_inv(d, N, limbs, 1, tables)
    assert np.array_equal(host(d), x)
    he.ntt_set_shape(N, 0, 0, 0)


def test_autotune_plan():
    pool = he.primes_generate(60, 1 << 16, 4)
    r = Rng(6)
    polys, keep = [], []
    for i, N in enumerate([4096, 32768, 8192, 16384, 4096, 32768]):
        t = he.NttTables(N, pool)
        x = r.uniform_limbs(pool[:1 + i % 4], N)
        d = dev(x)
        keep.append((t, x))
        polys.append((d, t, N, 1 + i % 4, 0))
    res = autotune.tune_plan(polys, reps=3, warmup=1)
    assert res["best"]["ok"] and len(res["candidates"]) == 2
    assert res["candidates"][0]["launches_per_direction"] == 1     # the mixed-degree launch
    for (d, _, _, _, _), (_, x) in zip(polys, keep):
        assert np.array_equal(host(d), x)                         # every candidate round-tripped


def test_autotune_mul_relin_rescale():
    N = 4096
    data, P = he.chain_primes(N, [60, 50, 50, 50], 60)
    ctx = he.Context(N, data, P)
    r = Rng(21)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    key = he.RelinKey(ctx, evk)
    res = autotune.tune_mul_relin_rescale(ctx, key, 3, 4, reps=2, warmup=1)
    assert res["log_thread_words"] in (3, 4) and all(c["ok"] for c in res["candidates"])
    # the chosen radix still matches the oracle
    ca = np.stack([r.uniform_limbs(data, N) for _ in range(2)])
    cb = np.stack([r.uniform_limbs(data, N) for _ in range(2)])
    out = torch.empty((1, 2, 3, N), dtype=torch.int64, device="cuda")
    he.mul_relin_rescale(out, dev(ca[None]), dev(cb[None]), 1, key, ctx, 3,
                         torch.empty(ctx.mrr_scratch_bytes(3, 1) // 8, dtype=torch.int64, device="cuda"))
    assert np.array_equal(host(out)[0], oracle.mul_relin_rescale(ca, cb, evk, data, P, 3))


def _small_server(**kw):
    args = dict(degrees=(4096, 8192), min_level=2, max_level=4, slots=4, streams=2, max_wait_s=0.001,
                pool_per_bucket=2, seed=11)
    args.update(kw)
    return serving.Server(**args)


_MODES = {"per_level": {}, "mixed_levels": {"mixed_levels": True}, "mixed_degrees": {"mixed_degrees": True}}


@pytest.mark.parametrize("mode", list(_MODES))
def test_serving_alone_equals_in_the_mix(mode):
    srv = _small_server(**_MODES[mode])
    reqs = srv.make_requests(240, rate=20000.0, seed=12)
    keep = [3, 50, 51, 52, 117, 200, 239]
    stats = srv.run(reqs, keep_ids=keep)
    assert stats["requests"] == 240 and len(srv.completed) == 240
    assert stats["batches"] < 240                      # requests were batched together
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    for rid in keep:
        alone = srv.serve_alone(reqs[rid])
        assert torch.equal(srv.keep[rid], alone), rid


@pytest.mark.parametrize("mode", list(_MODES))
def test_serving_result_matches_oracle(mode):
    degrees = (4096, 8192) if mode == "mixed_degrees" else (4096,)
    srv = _small_server(degrees=degrees, max_level=3, **_MODES[mode])
    reqs = srv.make_requests(20, rate=5000.0, seed=13)
    srv.run(reqs, keep_ids=[7])
    if mode != "per_level":   # one batch held several levels (and degrees)
        assert len({q.level for q in reqs}) > 1
    r = reqs[7]
    src = srv.pool[(r.N, r.level)][r.src].numpy().view(np.uint64)
    ctx = srv.ctx[r.N]
    # the server's keys are uniform words generated from its seed, degree by
    # degree; rebuild them
    rng = Rng(11)
    n_data = srv.max_level + 1
    for N in srv.degrees:
        data, P = srv.moduli[N], srv.ctx[N].P
        evk = np.stack([np.stack([rng.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(n_data)])
        if N == r.N:
            break
    data, P = srv.moduli[r.N], ctx.P
    ref = oracle.mul_relin_rescale(src[0], src[1], evk, data, P, r.level)
    assert np.array_equal(srv.keep[7].numpy().view(np.uint64).reshape(ref.shape), ref)


def test_serving_admission_respects_budget():
    srv = _small_server(slots=2)
    one_batch = sum(srv._batch_words(8192, 4, 2)) * 8
    srv.budget = srv.static_bytes + 2 * one_batch          # room for two open/in-flight batches
    reqs = srv.make_requests(60, rate=50000.0, seed=14)
    stats = srv.run(reqs)
    assert len(srv.completed) == 60
    assert srv.peak_ledger <= srv.budget
