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


@pytest.mark.parametrize("log_n", [10, 12, 15])
@pytest.mark.parametrize("offset_words", [0, 4])
def test_forward_store_forms(log_n, offset_words):
    """The forward transform of a uniform batch leaves by bulk tensor stores
    when the batch is 128-byte aligned and by plain stores otherwise (a
    32-byte aligned view 4 words into its buffer); both equal the oracle, and
    the words around the batch are untouched."""
    N = 1 << log_n
    limbs, count = 3, 3
    qs = _moduli(N, limbs)
    tables = he.NttTables(N, qs)
    x = np.stack([Rng(log_n * 100 + p).uniform_limbs(qs, N) for p in range(count)])
    buf = torch.full((count * limbs * N + 8,), 777, dtype=torch.int64, device="cuda")
    d = buf[offset_words:offset_words + count * limbs * N].view(count, limbs, N)
    assert d.data_ptr() % 128 == (0 if offset_words == 0 else 32)
    d.copy_(dev(x))
    he.ntt_fwd(d, N, limbs, count, tables)
    got = host(d)
    for p in range(count):
        assert np.array_equal(got[p], oracle.ntt_fwd(x[p], qs)), p
    rest = torch.cat([buf[:offset_words], buf[offset_words + count * limbs * N:]])
    assert bool((rest == 777).all().item())


SHAPES = [(10, 10, 3), (11, 11, 3), (11, 10, 4), (12, 12, 3), (12, 11, 4), (12, 10, 4), (13, 13, 4),
          (13, 12, 3), (13, 11, 4), (14, 13, 4), (14, 12, 3), (14, 12, 4), (15, 13, 4), (15, 12, 3),
          (15, 13, 3), (16, 13, 3), (16, 12, 4)]


@pytest.mark.parametrize("log_n,log_b,log_e", SHAPES)
def test_ntt_parity_alternate_shapes(log_n, log_b, log_e):
    """Every non-default kernel shape the autotuner may choose, through a
    plan (persistent launch), forward and inverse."""
    N = 1 << log_n
    qs = _moduli(N, 4)
    tables = he.NttTables(N, qs)
    x = np.stack([Rng(300 + log_b + 7 * log_e + p).uniform_limbs(qs, N) for p in range(3)])
    d = dev(x)
    plan = he.NttPlan([(d[p], tables, N, 4, 0) for p in range(3)], shapes={N: (log_b, log_e)})
    assert plan.launches == 1
    plan.fwd()
    got = host(d)
    for p in range(3):
        assert np.array_equal(got[p], oracle.ntt_fwd(x[p], qs))
    plan.inv()
    assert np.array_equal(host(d), x)


@pytest.mark.parametrize("log_n", [10, 11, 12, 13, 14, 15, 16])
def test_ntt_parity_every_tuner_candidate(log_n):
    """Every candidate the autotuner may apply -- each built shape (words per
    CTA, words per thread, CTAs per SM) launched as one cluster per limb and
    as a persistent grid -- through he_ntt_fwd / he_ntt_inv, against the
    oracle, with a ragged limb count."""
    N = 1 << log_n
    qs = _moduli(N, 3)
    tables = he.NttTables(N, qs)
    x = np.stack([Rng(700 + log_n + p).uniform_limbs(qs, N) for p in range(3)])
    ref = [oracle.ntt_fwd(x[p], qs) for p in range(3)]
    try:
        for lb, le, occ in he.ntt_shapes(N):
            for pers in (0, 1):
                he.ntt_set_shape(N, lb, le, pers, ctas_per_sm=occ)
                d = dev(x)
                he.ntt_fwd(d, N, 3, 3, tables)
                got = host(d)
                for p in range(3):
                    assert np.array_equal(got[p], ref[p]), (lb, le, occ, pers, p)
                he.ntt_inv(d, N, 3, 3, tables)
                assert np.array_equal(host(d), x), (lb, le, occ, pers)
    finally:
        he.ntt_set_shape(N, 0, 0, 0)


def test_mixed_degree_plan_single_launch():
    """Uneven batch (N from 2^12 to 2^15, 1 to 16 limbs from a pool of
    50-60-bit primes = 1 mod 2^16) in one launch per direction, with ragged
    limb counts that leave sub-clusters idle in the last unit of a degree."""
    pool = he.primes_generate(60, 1 << 16, 6) + he.primes_generate(55, 1 << 16, 5) + \
        he.primes_generate(50, 1 << 16, 5)
    tables = {N: he.NttTables(N, pool) for N in (4096, 8192, 16384, 32768)}
    r = Rng(3)
    Ns = [4096, 32768, 8192, 16384, 4096, 8192, 16384, 32768, 4096, 16384, 8192, 4096]
    limbs = [1, 3, 16, 5, 7, 2, 1, 1, 16, 3, 9, 4]
    firsts = [0, 2, 0, 11, 4, 14, 15, 5, 0, 1, 7, 12]
    polys = []
    for N, L, f in zip(Ns, limbs, firsts):
        polys.append(r.uniform_limbs(pool[f:f + L], N))
    d = [dev(x) for x in polys]
    plan = he.NttPlan([(d[i], tables[N], N, L, f) for i, (N, L, f) in enumerate(zip(Ns, limbs, firsts))])
    assert plan.launches == 1
    plan.fwd()
    for i, (N, L, f) in enumerate(zip(Ns, limbs, firsts)):
        assert np.array_equal(host(d[i]), oracle.ntt_fwd(polys[i], pool[f:f + L])), i
    plan.inv()
    for i in range(len(polys)):
        assert np.array_equal(host(d[i]), polys[i]), i


def test_per_degree_plan_with_shapes():
    """A plan with shape overrides runs one persistent launch per degree."""
    pool = he.primes_generate(60, 1 << 16, 3)
    tabs = {N: he.NttTables(N, pool) for N in (1024, 4096, 65536)}
    r = Rng(8)
    xs = [r.uniform_limbs(pool, N) for N in (1024, 4096, 65536)]
    ds = [dev(x) for x in xs]
    plan = he.NttPlan([(ds[i], tabs[N], N, 3, 0) for i, N in enumerate((1024, 4096, 65536))],
                      shapes={65536: (13, 3)})
    assert plan.launches == 3
    plan.fwd()
    for i in range(3):
        assert np.array_equal(host(ds[i]), oracle.ntt_fwd(xs[i], pool))
    plan.inv()
    for i in range(3):
        assert np.array_equal(host(ds[i]), xs[i])


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
