"""GPU parity of mixed-level MulLinRS batches (he_mul_relin_rescale_batch):
jobs of different levels and counts under one context run with one launch
per pipeline stage, and every output is bit-exact against the oracle and
equal to the single-level call on the same pair. Covers odd counts (a
partial two-ciphertext chunk in the key multiply-accumulate), jobs with
count 0, more than 16 jobs (a second pass), both evaluation shapes, and the
argument checks."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402

CHAINS = {
    "small4k": (4096, [60, 50, 50, 50, 50], 60),
    "ckks16k": (16384, [60] + [50] * 6, 60),
}


def _setup(name, seed):
    N, bits, pbits = CHAINS[name]
    data, P = he.chain_primes(N, bits, pbits)
    ctx = he.Context(N, data, P)
    r = Rng(seed)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    return N, data, P, ctx, evk, he.RelinKey(ctx, evk), r


def _cts(r, qs, N, count):
    if count == 0:
        return np.zeros((0, 2, len(qs), N), dtype=np.uint64)
    return np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(count)])


def _run(ctx, key, N, jobs_np):
    """Device batch of (ca, cb, level) host jobs; returns host outputs."""
    jobs, outs = [], []
    for ca, cb, level in jobs_np:
        count = len(ca)
        out = empty(max(count, 1), 2, level, N)
        outs.append(out)
        jobs.append((out, dev(ca) if count else empty(1, 2, level + 1, N),
                     dev(cb) if count else empty(1, 2, level + 1, N), count, level))
    sc = empty(max(8, ctx.mrr_batch_scratch_bytes(jobs) // 8))
    he.mul_relin_rescale_batch(jobs, key, ctx, sc)
    return [host(o) for o in outs]


@pytest.mark.parametrize("log_e", [4, 3])
def test_mixed_levels_against_oracle(log_e):
    N, data, P, ctx, evk, key, r = _setup("small4k", 40 + log_e)
    ctx.set_eval_shape(log_e)
    spec = [(3, 4), (1, 1), (2, 3), (0, 2), (5, 2), (1, 4)]
    jobs = []
    for count, level in spec:
        qs = data[:level + 1]
        jobs.append((_cts(r, qs, N, count), _cts(r, qs, N, count), level))
    got = _run(ctx, key, N, jobs)
    for (ca, cb, level), g in zip(jobs, got):
        for c in range(len(ca)):
            assert np.array_equal(g[c], oracle.mul_relin_rescale(ca[c], cb[c], evk, data, P, level)), (level, c)


def test_mixed_levels_equal_single_calls_at_benchmark_size():
    """N = 2^14 with the 60 + 6 x 50-bit chain, every level 1..6 in one batch
    (uneven counts), against he_mul_relin_rescale per level; two pairs of the
    level-6 job also against the oracle."""
    N, data, P, ctx, evk, key, r = _setup("ckks16k", 50)
    spec = [(6, 6), (3, 1), (1, 2), (4, 3), (2, 4), (7, 5)]
    jobs = []
    for count, level in spec:
        qs = data[:level + 1]
        jobs.append((_cts(r, qs, N, count), _cts(r, qs, N, count), level))
    got = _run(ctx, key, N, jobs)
    for (ca, cb, level), g in zip(jobs, got):
        count = len(ca)
        out = empty(count, 2, level, N)
        he.mul_relin_rescale(out, dev(ca), dev(cb), count, key, ctx, level,
                             empty(ctx.mrr_scratch_bytes(level, count) // 8))
        assert np.array_equal(g, host(out)), level
    ca, cb, level = jobs[0]
    for c in (0, len(ca) - 1):
        assert np.array_equal(got[0][c], oracle.mul_relin_rescale(ca[c], cb[c], evk, data, P, level))


def test_more_jobs_than_one_pass():
    """18 jobs (the job table holds 16): the batch runs in two passes."""
    N, data, P, ctx, evk, key, r = _setup("small4k", 60)
    jobs = []
    for i in range(18):
        level = 1 + i % 4
        qs = data[:level + 1]
        jobs.append((_cts(r, qs, N, 1 + i % 3), _cts(r, qs, N, 1 + i % 3), level))
    got = _run(ctx, key, N, jobs)
    for (ca, cb, level), g in zip(jobs, got):
        out = empty(len(ca), 2, level, N)
        he.mul_relin_rescale(out, dev(ca), dev(cb), len(ca), key, ctx, level,
                             empty(ctx.mrr_scratch_bytes(level, len(ca)) // 8))
        assert np.array_equal(g, host(out))


def test_batch_argument_checks():
    N, data, P, ctx, evk, key, r = _setup("small4k", 70)
    a, out = empty(2, 2, 3, N), empty(2, 2, 2, N)
    sc = empty(ctx.mrr_batch_scratch_bytes([(2, 2)]) // 8)
    he.mul_relin_rescale_batch([], key, ctx, sc)                       # nothing to do
    he.mul_relin_rescale_batch([(out, a, a, 0, 2)], key, ctx, sc)      # count 0
    with pytest.raises(he.HeError):
        he.mul_relin_rescale_batch([(out, a, a, 2, 0)], key, ctx, sc)  # level 0 cannot rescale
    with pytest.raises(he.HeError):
        he.mul_relin_rescale_batch([(out, a, a, 2, 2)], key, ctx, sc[:16])   # short scratch
    assert ctx.mrr_batch_scratch_bytes([(2, 2)]) == 2 * (2 + 3) ** 2 * N * 8
    assert ctx.mrr_batch_scratch_bytes([(2, 9)]) == 0                  # level beyond the chain
