"""GPU parity of the negacyclic NTT (Sec. II-B, Sec. III-B) and the dyadic
product through the C ABI: bit-exact against the CPU oracle on the same
seeded inputs, at every supported degree, on batches that span many CTAs and
clusters with ragged limb counts, at the full 1024 x 8 x 2^15 workload
(sampled limbs), and on edge values."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng
from tests import bruteforce as bf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402


def _moduli(N, k, seed=0):
    two_n = 2 * N
    qs = he.primes_generate(60, two_n, (k + 1) // 2) + he.primes_generate(50, two_n, k // 2)
    return qs[:k]


@pytest.mark.parametrize("log_n", list(range(10, 17)))
def test_ntt_parity_every_degree(log_n):
    N = 1 << log_n
    limbs, count = 3, 2                       # 6 limbs, ragged against clusters
    qs = _moduli(N, limbs)
    tables = he.NttTables(N, qs)
    for l, q in enumerate(qs):
        assert tables.psi(l) == oracle.find_psi(q, N)
    x = np.stack([Rng(log_n * 10 + p).uniform_limbs(qs, N) for p in range(count)])
    d = dev(x)
    he.ntt_fwd(d, N, limbs, count, tables)
    got = host(d)
    for p in range(count):
        assert np.array_equal(got[p], oracle.ntt_fwd(x[p], qs)), p
    he.ntt_inv(d, N, limbs, count, tables)
    assert np.array_equal(host(d), x)
    # inverse on independent NTT-domain input
    y = np.stack([Rng(log_n * 10 + 7 + p).uniform_limbs(qs, N) for p in range(count)])
    dy = dev(y)
    he.ntt_inv(dy, N, limbs, count, tables)
    got = host(dy)
    for p in range(count):
        assert np.array_equal(got[p], oracle.ntt_inv(y[p], qs)), p


@pytest.mark.parametrize("log_n,log_b", [(12, 11), (12, 10), (13, 13), (13, 11), (14, 13), (14, 11), (15, 13),
                                         (11, 10)])
def test_ntt_parity_alternate_shapes(log_n, log_b):
    """Every kernel shape the autotuner may choose, through a plan."""
    N = 1 << log_n
    qs = _moduli(N, 4)
    tables = he.NttTables(N, qs)
    x = np.stack([Rng(300 + log_b + p).uniform_limbs(qs, N) for p in range(3)])
    d = dev(x)
    plan = he.NttPlan([(d[p], tables, N, 4, 0) for p in range(3)], shapes={N: log_b})
    plan.fwd()
    got = host(d)
    for p in range(3):
        assert np.array_equal(got[p], oracle.ntt_fwd(x[p], qs))
    plan.inv()
    assert np.array_equal(host(d), x)


def test_ntt_edge_values():
    N = 1 << 15
    qs = _moduli(N, 2)
    tables = he.NttTables(N, qs)
    cases = [np.zeros((2, N), np.uint64),
             np.stack([np.full(N, q - 1, np.uint64) for q in qs]),
             np.stack([np.where(np.arange(N) % 2 == 0, q - 1, 0).astype(np.uint64) for q in qs])]
    one = np.zeros((2, N), np.uint64)
    one[:, 0] = 1
    cases.append(one)
    for x in cases:
        d = dev(x)
        he.ntt_fwd(d, N, 2, 1, tables)
        got = host(d)
        assert np.array_equal(got, oracle.ntt_fwd(x, qs))
        he.ntt_inv(d, N, 2, 1, tables)
        assert np.array_equal(host(d), x)
    assert (oracle.ntt_fwd(one, qs) == 1).all()


def test_plain_workload_against_schoolbook():
    """N = 4096, two 60-bit primes (seed 1): NTT, dyadic product and inverse
    NTT on the GPU equal the O(N^2) negacyclic convolution."""
    N = 4096
    qs = he.primes_generate(60, 2 * N, 2)
    tables = he.NttTables(N, qs)
    r = Rng(1)
    a, b = r.uniform_limbs(qs, N), r.uniform_limbs(qs, N)
    da, db = dev(a), dev(b)
    he.ntt_fwd(da, N, 2, 1, tables)
    he.ntt_fwd(db, N, 2, 1, tables)
    dc = empty(2, N)
    he.dyadic_mul(dc, da, db, N, 2, 1, tables)
    he.ntt_inv(dc, N, 2, 1, tables)
    c = host(dc)
    for l, q in enumerate(qs):
        assert [int(v) for v in c[l]] == bf.negacyclic_schoolbook(a[l], b[l], q)


@pytest.mark.parametrize("N,limbs,count", [(4096, 2, 3), (16384, 7, 2), (32768, 5, 1)])
def test_dyadic_parity(N, limbs, count):
    qs = _moduli(N, limbs)
    tables = he.NttTables(N, qs)
    r = Rng(N + limbs)
    a = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    b = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    # adversarial values: largest residues
    a[0, :, :4] = np.array(qs, dtype=np.uint64)[:, None] - 1
    b[0, :, :4] = np.array(qs, dtype=np.uint64)[:, None] - 1
    da, db, dc = dev(a), dev(b), empty(count, limbs, N)
    he.dyadic_mul(dc, da, db, N, limbs, count, tables)
    got = host(dc)
    for p in range(count):
        assert np.array_equal(got[p], oracle.dyadic(a[p], b[p], qs))


def test_naive_baseline_parity():
    N = 1 << 14
    qs = _moduli(N, 3)
    tables = he.NttTables(N, qs)
    x = np.stack([Rng(77 + p).uniform_limbs(qs, N) for p in range(2)])
    d = dev(x)
    he.ntt_fwd_naive(d, N, 3, 2, tables)
    got = host(d)
    for p in range(2):
        assert np.array_equal(got[p], oracle.ntt_fwd(x[p], qs))
    he.ntt_inv_naive(d, N, 3, 2, tables)
    assert np.array_equal(host(d), x)


def test_full_workload_sampled():
    """The benchmark workload (1024 instances x 8 limbs at N = 2^15, one
    launch per direction as the benchmark runs it), checked on sampled limbs
    against the oracle and on all limbs by the exact round trip."""
    N, limbs, count = 1 << 15, 8, 1024
    qs = he.primes_generate(60, 2 * N, 4) + he.primes_generate(50, 2 * N, 4)
    tables = he.NttTables(N, qs)
    r = Rng(15)
    x = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    d = dev(x)
    he.ntt_fwd(d, N, limbs, count, tables)
    got = host(d)
    for p, l in [(0, 0), (0, 7), (511, 3), (1023, 7), (700, 1)]:
        assert np.array_equal(got[p, l], oracle.ntt_fwd(x[p, l:l + 1], [qs[l]])[0]), (p, l)
    assert (got < np.array(qs, dtype=np.uint64)[None, :, None]).all()
    he.ntt_inv(d, N, limbs, count, tables)
    assert np.array_equal(host(d), x)
