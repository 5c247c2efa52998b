"""GPU parity of the multi-degree MulLinRS batch (Sec. IV-C routine, batched
over instances of different degrees as in Sec. III-B): one launch per
pipeline stage for jobs of N = 2^12 .. 2^15, each under its own context and
key, levels and counts mixed. Every output equals the per-degree
he_mul_relin_rescale call bit for bit, and sampled jobs equal the oracle."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402

_CACHE = {}


def _chain(N, n_data):
    """Context and key of degree N: 60-bit q_0, 50-bit q_1.., 60-bit P (the
    serving chains); the key is uniform (pseudo-random like a real key)."""
    if (N, n_data) not in _CACHE:
        data, P = he.chain_primes(N, [60] + [50] * (n_data - 1), 60)
        ctx = he.Context(N, data, P)
        r = Rng(900 + N + n_data)
        evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(n_data)])
        _CACHE[(N, n_data)] = (data, P, ctx, evk, he.RelinKey(ctx, evk))
    return _CACHE[(N, n_data)]


def _jobs(spec, seed):
    """spec: list of (N, n_data, level, count) -> device jobs + host inputs."""
    r = Rng(seed)
    jobs, host_in = [], []
    for N, n_data, level, count in spec:
        data, P, ctx, evk, key = _chain(N, n_data)
        qs = data[:level + 1]
        a = np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(count)]) if count else \
            np.zeros((0, 2, level + 1, N), dtype=np.uint64)
        b = np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(count)]) if count else \
            np.zeros((0, 2, level + 1, N), dtype=np.uint64)
        da = dev(a) if count else empty(2)
        db = dev(b) if count else empty(2)
        out = empty(max(count, 1), 2, level, N)
        jobs.append((out, da, db, count, level, key, ctx))
        host_in.append((a, b))
    return jobs, host_in


def _per_degree(job):
    out, da, db, count, level, key, ctx = job
    ref = empty(count, 2, level, ctx.N)
    he.mul_relin_rescale(ref, da, db, count, key, ctx, level, empty(ctx.mrr_scratch_bytes(level, count) // 8))
    return host(ref)


SPEC_MIXED = [(8192, 4, 2, 3), (32768, 4, 3, 1), (4096, 4, 1, 5), (16384, 4, 3, 2), (8192, 4, 3, 0),
              (16384, 4, 1, 7), (4096, 4, 3, 1), (32768, 4, 1, 2)]


def test_multi_degree_batch_equals_per_degree_and_oracle():
    jobs, host_in = _jobs(SPEC_MIXED, 31)
    scratch = empty(he.mul_relin_rescale_multi_scratch_bytes([(j[3], j[4], j[5], j[6]) for j in jobs]) // 8)
    he.mul_relin_rescale_multi(jobs, scratch)
    got = [host(j[0]) for j in jobs]
    for i, job in enumerate(jobs):
        count = job[3]
        if not count:
            continue
        assert np.array_equal(got[i][:count], _per_degree(job)), i
    # sampled pairs of every degree against the oracle
    for i in (0, 1, 2, 3):
        out, da, db, count, level, key, ctx = jobs[i]
        data, P, _, evk, _ = _chain(ctx.N, 4)
        a, b = host_in[i]
        for c in {0, count - 1}:
            assert np.array_equal(got[i][c], oracle.mul_relin_rescale(a[c], b[c], evk, data, P, level)), (i, c)


def test_multi_degree_serving_mix_levels_2_to_16():
    """The serving mix: N in {2^13, 2^14, 2^15}, levels 2..16 (17 data
    primes + P per degree), one pair per job, 18 jobs (two passes)."""
    levels = [2, 16, 7, 11, 3, 14, 5, 9, 16, 2, 12, 6, 15, 4, 10, 8, 13, 3]
    degs = [8192, 16384, 32768] * 6
    spec = [(N, 17, lv, 1) for N, lv in zip(degs, levels)]
    jobs, host_in = _jobs(spec, 32)
    scratch = empty(he.mul_relin_rescale_multi_scratch_bytes([(j[3], j[4], j[5], j[6]) for j in jobs]) // 8)
    he.mul_relin_rescale_multi(jobs, scratch)
    for i, job in enumerate(jobs):
        assert np.array_equal(host(job[0]), _per_degree(job)), i
    # the oracle on the smallest job of each degree
    for i in (0, 9, 13):
        out, da, db, count, level, key, ctx = jobs[i]
        data, P, _, evk, _ = _chain(ctx.N, 17)
        a, b = host_in[i]
        assert np.array_equal(host(out)[0], oracle.mul_relin_rescale(a[0], b[0], evk, data, P, level)), i


def test_multi_degree_repeated_calls_and_graph_safe_inputs():
    """Two calls in a row on new inputs give new, correct outputs (no state
    carried between calls in the scratch)."""
    for seed in (33, 34):
        jobs, _ = _jobs([(4096, 3, 2, 2), (32768, 3, 2, 1), (8192, 3, 1, 3)], seed)
        scratch = empty(he.mul_relin_rescale_multi_scratch_bytes([(j[3], j[4], j[5], j[6]) for j in jobs]) // 8)
        scratch.fill_(-1)
        he.mul_relin_rescale_multi(jobs, scratch)
        for i, job in enumerate(jobs):
            assert np.array_equal(host(job[0]), _per_degree(job)), (seed, i)


def test_multi_degree_argument_checks():
    jobs, _ = _jobs([(4096, 3, 2, 1), (8192, 3, 2, 1)], 35)
    need = he.mul_relin_rescale_multi_scratch_bytes([(j[3], j[4], j[5], j[6]) for j in jobs])
    with pytest.raises(he.HeError, match="scratch too small"):
        he.mul_relin_rescale_multi(jobs, empty(need // 8 - 1))
    # a key of another context
    bad = list(jobs[0])
    bad[5] = _chain(8192, 3)[4]
    with pytest.raises(he.HeError, match="key"):
        he.mul_relin_rescale_multi([tuple(bad)], empty(need // 8))
    # a level without a limb to rescale away
    bad = list(jobs[0])
    bad[4] = 0
    with pytest.raises(he.HeError):
        he.mul_relin_rescale_multi([tuple(bad)], empty(need // 8))
    # degrees outside 2^12 .. 2^15
    data, P = he.chain_primes(2048, [60, 50, 50], 60)
    ctx = he.Context(2048, data, P)
    r = Rng(36)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], 2048) for _ in range(2)]) for _ in range(3)])
    key = he.RelinKey(ctx, evk)
    small = (empty(2, 1, 2048), empty(2, 2, 2048), empty(2, 2, 2048), 1, 1, key, ctx)
    with pytest.raises(he.HeError, match="outside"):
        he.mul_relin_rescale_multi([small], empty(need // 8))
    assert he.mul_relin_rescale_multi_scratch_bytes([(1, 1, key, ctx)]) == 0
    # count-0 jobs alone: nothing to do, nothing written
    zero = (empty(1), empty(2), empty(2), 0, 2, jobs[0][5], jobs[0][6])
    he.mul_relin_rescale_multi([zero], empty(1))
