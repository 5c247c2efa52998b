"""Pins for the oracle's multi-threaded runners (they time the CPU baseline):
each unit (polynomial, limb) must be transformed with its own limb's modulus,
and the batch result must not depend on the thread count. The runners are
checked against the defining sum of the negacyclic NTT (Sec. II-B) evaluated
directly, against the single-polynomial oracle calls, and the MulLinRS runner
against the per-pair oracle routine (Sec. II-A)."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300.synth import Rng
from tests import bruteforce as bf


def _mixed_moduli(N):
    # distinct sizes, so that a limb paired with another limb's modulus gives
    # a different (usually out-of-range) result
    return (oracle.find_primes(60, 2 * N, 2) + oracle.find_primes(50, 2 * N, 1)
            + oracle.find_primes(40, 2 * N, 1))


def _batch(qs, N, polys, seed):
    r = Rng(seed)
    return np.stack([r.uniform_limbs(qs, N) for _ in range(polys)])


@pytest.mark.parametrize("threads", [1, 4])
def test_ntt_fwd_many_equals_definition(threads):
    N = 64
    qs = _mixed_moduli(N)
    x = _batch(qs, N, 3, 41)
    X = oracle.ntt_fwd_many(x, qs, threads)
    assert X.shape == x.shape and X.dtype == np.uint64
    for p in range(x.shape[0]):
        for l, q in enumerate(qs):
            assert [int(v) for v in X[p, l]] == bf.ntt_definition(x[p, l], q, oracle.find_psi(q, N))


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_ntt_many_equal_per_row_calls(threads):
    N = 1024
    qs = _mixed_moduli(N)
    x = _batch(qs, N, 5, 42)
    X = oracle.ntt_fwd_many(x, qs, threads)
    Y = _batch(qs, N, 5, 43)          # independent NTT-domain input for the inverse
    y = oracle.ntt_inv_many(Y, qs, threads)
    for p in range(x.shape[0]):
        assert np.array_equal(X[p], oracle.ntt_fwd(x[p], qs))
        assert np.array_equal(y[p], oracle.ntt_inv(Y[p], qs))
    # the inputs are left untouched (the runners work on copies) and the two
    # runners invert each other
    assert np.array_equal(oracle.ntt_inv_many(X, qs, threads), x)
    assert np.array_equal(x, _batch(qs, N, 5, 42))


def test_ntt_many_sensitive_to_limb_modulus_pairing():
    """A runner that paired limb l with another limb's modulus would fail
    the checks above: the rows differ under the swapped pairing."""
    N = 256
    qs = _mixed_moduli(N)
    x = _batch(qs, N, 1, 44)
    X = oracle.ntt_fwd_many(x, qs, 2)
    for l in range(len(qs)):
        other = qs[(l + 1) % len(qs)]
        wrong = oracle.ntt_fwd(x[0, l:l + 1] % np.uint64(other), [other])[0]
        assert not np.array_equal(X[0, l], wrong)


@pytest.mark.parametrize("threads", [1, 3])
def test_mul_relin_rescale_many_equals_per_pair(threads):
    N = 64
    data = [oracle.find_primes(60, 2 * N, 1)[0]] + oracle.find_primes(50, 2 * N, 3)
    P = oracle.find_primes(60, 2 * N, 2)[1]
    n_max = len(data)
    r = Rng(45)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(n_max)])
    for level in (1, 3):
        qs = data[:level + 1]
        cts_a = [np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(4)]
        cts_b = [np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(4)]
        got = oracle.mul_relin_rescale_many(cts_a, cts_b, evk, data, P, level, threads)
        assert len(got) == 4
        for i in range(4):
            ref = oracle.mul_relin_rescale(cts_a[i], cts_b[i], evk, data, P, level)
            assert got[i].shape == (2, level, N)
            assert np.array_equal(got[i], ref)
