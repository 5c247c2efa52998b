"""GPU parity of the fused negacyclic product (he_negacyclic_mul: forward
transforms of a and b, pointwise product and inverse transform in one
launch, Sec. II-B): bit-exact against the oracle's product at every degree
and in every built transform shape, against the O(N^2) schoolbook
convolution on the plain workload (N = 4096, two 60-bit primes), in place,
on a large batch (sampled), and with the argument checks."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng
from tests import bruteforce as bf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402


def _moduli(N, k):
    qs = he.primes_generate(60, 2 * N, (k + 1) // 2) + he.primes_generate(50, 2 * N, k // 2)
    return qs[:k]


def _check(N, limbs, count, seed):
    qs = _moduli(N, limbs)
    tables = he.NttTables(N, qs)
    r = Rng(seed)
    a = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    b = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    c = empty(count, limbs, N)
    he.negacyclic_mul(c, dev(a), dev(b), N, limbs, count, tables)
    got = host(c)
    for p in range(count):
        assert np.array_equal(got[p], oracle.negacyclic_mul(a[p], b[p], qs)), p


@pytest.mark.parametrize("log_n", list(range(10, 17)))
def test_every_degree(log_n):
    _check(1 << log_n, 3, 2, 500 + log_n)


@pytest.mark.parametrize("log_n", [12, 14, 15, 16])
def test_every_shape(log_n):
    """The product runs in the forward transform's configured shape: every
    shape built for the degree."""
    N = 1 << log_n
    try:
        for lb, le, occ in he.ntt_shapes(N):
            he.ntt_set_shape(N, lb, le, direction=he.FORWARD, ctas_per_sm=occ)
            _check(N, 2, 2, 600 + lb + 7 * le + 13 * occ)
    finally:
        he.ntt_set_shape(N, 0, 0, direction=he.FORWARD)


def test_plain_workload_against_schoolbook():
    N = 4096
    qs = he.primes_generate(60, 2 * N, 2)
    tables = he.NttTables(N, qs)
    r = Rng(1)
    a, b = r.uniform_limbs(qs, N), r.uniform_limbs(qs, N)
    dc = empty(2, N)
    he.negacyclic_mul(dc, dev(a), dev(b), N, 2, 1, tables)
    c = host(dc)
    for l, q in enumerate(qs):
        assert [int(v) for v in c[l]] == bf.negacyclic_schoolbook(a[l], b[l], q)


def test_in_place_and_edges():
    N, limbs = 8192, 3
    qs = _moduli(N, limbs)
    tables = he.NttTables(N, qs)
    r = Rng(700)
    a, b = r.uniform_limbs(qs, N), r.uniform_limbs(qs, N)
    a[:, :4] = np.array([[0, 1, q - 1, q - 2] for q in qs], dtype=np.uint64)
    ref = oracle.negacyclic_mul(a, b, qs)
    da, db = dev(a), dev(b)
    he.negacyclic_mul(da, da, db, N, limbs, 1, tables)          # c = a
    assert np.array_equal(host(da), ref)
    da = dev(a)
    he.negacyclic_mul(db, da, db, N, limbs, 1, tables)          # c = b
    assert np.array_equal(host(db), ref)
    he.negacyclic_mul(empty(1), da, da, N, limbs, 0, tables)    # count 0
    big = empty(2, limbs, N).view(-1)
    with pytest.raises(he.HeError):                             # c overlaps a, unequal
        he.negacyclic_mul(big[N:], big, big, N, limbs, 1, tables)


def test_large_batch_sampled():
    """128 polynomials x 8 limbs at N = 2^15 in one launch; four polynomials
    checked against the oracle."""
    N, limbs, count = 32768, 8, 128
    qs = _moduli(N, limbs)
    tables = he.NttTables(N, qs)
    r = Rng(800)
    a = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    b = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    c = empty(count, limbs, N)
    he.negacyclic_mul(c, dev(a), dev(b), N, limbs, count, tables)
    got = host(c)
    for p in (0, 1, 77, count - 1):
        assert np.array_equal(got[p], oracle.negacyclic_mul(a[p], b[p], qs)), p
