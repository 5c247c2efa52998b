"""GPU parity of the other evaluation routines (Sec. IV-C: MulLin, SqrLinRS)
and of the encrypted matrix product C += A B (Sec. IV-E matMul_mxnxk, with
one relinearization per output), bit-exact against the oracle on the same
seeded inputs; plus decoded slots of a real encrypted matrix product against
numpy's product of the plaintext slot matrices."""
import numpy as np
import pytest

import oracle
from oracle import ckks
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402

CHAINS = {
    "small4k": (4096, [60, 50, 50, 50], 60),
    "matrix8k": (8192, [60, 40, 40], 60),
}


def _setup(name, seed):
    N, bits, pbits = CHAINS[name]
    data, P = he.chain_primes(N, bits, pbits)
    ctx = he.Context(N, data, P)
    r = Rng(seed)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    return N, data, P, ctx, evk, he.RelinKey(ctx, evk), r


def _cts(r, qs, N, count, comps=2):
    return np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(comps)]) for _ in range(count)])


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("name,level,count", [("small4k", 3, 3), ("small4k", 0, 2), ("matrix8k", 2, 5)])
def test_mul_relin(name, level, count, fused):
    N, data, P, ctx, evk, key, r = _setup(name, 70 + level + count)
    qs = data[:level + 1]
    ca, cb = _cts(r, qs, N, count), _cts(r, qs, N, count)
    out = empty(count, 2, level + 1, N)
    n = level + 1
    nbytes = (3 * n + 2) * N * 8 * count if fused else ctx.mul_relin_scratch_bytes(level, count)
    he.mul_relin(out, dev(ca), dev(cb), count, key, ctx, level, empty(nbytes // 8))
    got = host(out)
    for c in range(count):
        assert np.array_equal(got[c], oracle.relin(oracle.tensor(ca[c], cb[c], qs), evk, data, P, level)), c


@pytest.mark.parametrize("name,level,count", [("small4k", 3, 4), ("matrix8k", 2, 3)])
def test_sqr_relin_rescale(name, level, count):
    N, data, P, ctx, evk, key, r = _setup(name, 80 + level)
    qs = data[:level + 1]
    ca = _cts(r, qs, N, count)
    out = empty(count, 2, level, N)
    he.sqr_relin_rescale(out, dev(ca), count, key, ctx, level, empty(ctx.mrr_scratch_bytes(level, count) // 8))
    got = host(out)
    for c in range(count):
        assert np.array_equal(got[c], oracle.mul_relin_rescale(ca[c], ca[c], evk, data, P, level)), c


@pytest.mark.parametrize("fused", [False, True])
def test_relin_rescale_of_three_component_inputs(fused):
    N, data, P, ctx, evk, key, r = _setup("small4k", 90)
    level, count = 3, 3
    qs = data[:level + 1]
    c3 = _cts(r, qs, N, count, 3)
    out = empty(count, 2, level, N)
    nbytes = (3 * (level + 1) + 4) * N * 8 * count if fused else ctx.mrr_scratch_bytes(level, count)
    he.relin_rescale(out, dev(c3), count, key, ctx, level, empty(nbytes // 8))
    got = host(out)
    for c in range(count):
        ref = oracle.rescale(oracle.relin(c3[c], evk, data, P, level), data, level)
        assert np.array_equal(got[c], ref), c


@pytest.mark.parametrize("components", [2, 3])
def test_ct_add_and_in_place(components):
    N, data, P, ctx, evk, key, r = _setup("small4k", 95)
    level, count = 2, 3
    qs = data[:level + 1]
    a, b = _cts(r, qs, N, count, components), _cts(r, qs, N, count, components)
    da, db = dev(a), dev(b)
    out = empty(count, components, level + 1, N)
    he.ct_add(out, da, db, count, components, ctx, level)
    ref = np.stack([oracle.add(a[c], b[c], qs) for c in range(count)])
    assert np.array_equal(host(out), ref)
    he.ct_add(da, da, db, count, components, ctx, level)        # in place
    assert np.array_equal(host(da), ref)


@pytest.mark.parametrize("m,k,n", [(3, 2, 5), (1, 3, 1), (4, 4, 4), (2, 1, 9)])
def test_matmul_tensor(m, k, n):
    """Odd column counts leave a partial tile of output columns."""
    N, data, P, ctx, evk, key, r = _setup("small4k", 100 + m * 16 + k * 4 + n)
    level = 1
    qs = data[:level + 1]
    A = np.stack([_cts(r, qs, N, k) for _ in range(m)])
    B = np.stack([_cts(r, qs, N, n) for _ in range(k)])
    T = empty(m, n, 3, level + 1, N)
    he.ct_matmul_tensor(T, dev(A), dev(B), m, k, n, ctx, level)
    assert np.array_equal(host(T), oracle.matmul_tensor(A, B, qs))


def test_encrypted_matrix_product_accumulates_into_c():
    """C += A B with lazy relinearization: tensor, one relin + rescale per
    output, add into C; limbs equal the oracle composition, decoded slots
    equal the slot-wise matrix product plus C's own slots."""
    N, bits, pbits = CHAINS["matrix8k"]
    data, P = oracle.chain_primes(N, bits, pbits)
    r = Rng(5)
    keys = ckks.keygen(N, data, P, r)
    ctx = he.Context(N, data, P)
    key = he.RelinKey(ctx, keys.evk)
    scale = 2.0 ** 40
    m, k, n, L = 2, 3, 2, len(data) - 1
    zA = np.array([[r.complex_slots(N // 2) for _ in range(k)] for _ in range(m)])
    zB = np.array([[r.complex_slots(N // 2) for _ in range(n)] for _ in range(k)])
    zC = np.array([[r.complex_slots(N // 2) for _ in range(n)] for _ in range(m)])
    enc = lambda z, s, lvl=None: ckks.encrypt(ckks.encode_real(z, N, s), keys, r, level=lvl)
    A = np.stack([np.stack([enc(zA[i, l], scale) for l in range(k)]) for i in range(m)])
    B = np.stack([np.stack([enc(zB[l, j], scale) for j in range(n)]) for l in range(k)])
    out_scale = scale * scale / data[L]
    C = np.stack([np.stack([enc(zC[i, j], out_scale, L - 1) for j in range(n)]) for i in range(m)])
    T = empty(m, n, 3, L + 1, N)
    he.ct_matmul_tensor(T, dev(A), dev(B), m, k, n, ctx, L)
    R = empty(m * n, 2, L, N)
    he.relin_rescale(R, T, m * n, key, ctx, L, empty(ctx.mrr_scratch_bytes(L, m * n) // 8))
    dC = dev(C)
    he.ct_add(dC, dC, R, m * n, 2, ctx, L - 1)
    got = host(dC).reshape(m, n, 2, L, N)
    Tref = oracle.matmul_tensor(A, B, data)
    for i in range(m):
        for j in range(n):
            ref = oracle.add(C[i, j], oracle.rescale(oracle.relin(Tref[i, j], keys.evk, data, P, L), data, L),
                             data[:L])
            assert np.array_equal(got[i, j], ref), (i, j)
            z = ckks.decrypt_decode(got[i, j], keys, out_scale)
            exact = zC[i, j] + sum(zA[i, l] * zB[l, j] for l in range(k))
            assert float(np.abs(z - exact).max() / max(1.0, np.abs(exact).max())) < 1e-5


def test_matmul_tensor_moduli_below_2_32():
    """31-bit moduli take the per-term reduction path of the kernel."""
    N = 4096
    data = he.primes_generate(31, 2 * N, 2)
    P = he.primes_generate(32, 2 * N, 1)[0]
    ctx = he.Context(N, data, P)
    r = Rng(131)
    m, k, n, level = 2, 5, 3, 1
    A = np.stack([_cts(r, data, N, k) for _ in range(m)])
    B = np.stack([_cts(r, data, N, n) for _ in range(k)])
    T = empty(m, n, 3, level + 1, N)
    he.ct_matmul_tensor(T, dev(A), dev(B), m, k, n, ctx, level)
    assert np.array_equal(host(T), oracle.matmul_tensor(A, B, data))


@pytest.mark.parametrize("g_kind", ["rot1", "rot7", "conj"])
def test_ct_automorph_matches_coefficient_domain(g_kind):
    N, data, P, ctx, evk, key, r = _setup("small4k", 140)
    level, count = 2, 2
    qs = data[:level + 1]
    g = {"rot1": 5, "rot7": pow(5, 7, 2 * N), "conj": 2 * N - 1}[g_kind]
    ct = _cts(r, qs, N, count)
    out = empty(count, 2, level + 1, N)
    he.ct_automorph(out, dev(ct), count, 2, g, ctx, level)
    got = host(out)
    for c in range(count):
        for k in range(2):
            assert np.array_equal(got[c, k], oracle.ntt_automorphism(ct[c, k], g, qs)), (c, k)


@pytest.mark.parametrize("fused", [False, True])
def test_rotate_matches_oracle(fused):
    N, data, P, ctx, evk, key, r = _setup("small4k", 150)
    level, count, g = 3, 3, pow(5, 3, 2 * 4096)
    qs = data[:level + 1]
    ct = _cts(r, qs, N, count)
    out = empty(count, 2, level + 1, N)
    n = level + 1
    nbytes = (3 * n + 3 * n + 2) * N * 8 * count if fused else ctx.rotate_scratch_bytes(level, count)
    he.rotate(out, dev(ct), count, g, key, ctx, level, empty(nbytes // 8))   # evk serves as the Galois key
    got = host(out)
    for c in range(count):
        assert np.array_equal(got[c], oracle.rotate(ct[c], g, evk, data, P, level)), c


def test_rotate_real_encryption_rolls_slots():
    N, bits, pbits = CHAINS["matrix8k"]
    data, P = oracle.chain_primes(N, bits, pbits)
    r = Rng(6)
    keys = ckks.keygen(N, data, P, r)
    k = 5
    g = pow(5, k, 2 * N)
    gk = ckks.galois_key(keys, g, r)
    ctx = he.Context(N, data, P)
    gkey = he.RelinKey(ctx, gk)
    scale, L = 2.0 ** 40, len(data) - 1
    z = r.complex_slots(N // 2)
    ct = ckks.encrypt(ckks.encode_real(z, N, scale), keys, r)
    out = empty(1, 2, L + 1, N)
    he.rotate(out, dev(ct[None]), 1, g, gkey, ctx, L, empty(ctx.rotate_scratch_bytes(L, 1) // 8))
    got = host(out)[0]
    assert np.array_equal(got, oracle.rotate(ct, g, gk, data, P, L))
    zr = ckks.decrypt_decode(got, keys, scale)
    assert float(np.abs(zr - np.roll(z, -k)).max()) < 1e-5


def test_full_size_matrix_product_sampled():
    """C += A B at 32 x 32 x 32, N = 8192, 60/40/40 + 60 (the benchmark's
    launch configuration): three sampled outputs against the oracle."""
    N, data, P, ctx, evk, key, r = _setup("matrix8k", 160)
    m = k = n = 32
    L = len(data) - 1
    A = np.stack([_cts(r, data, N, k) for _ in range(m)])
    B = np.stack([_cts(r, data, N, n) for _ in range(k)])
    C = np.stack([_cts(r, data[:L], N, n) for _ in range(m)])
    T = empty(m * n, 3, L + 1, N)
    he.ct_matmul_tensor(T, dev(A), dev(B), m, k, n, ctx, L)
    R = empty(m * n, 2, L, N)
    he.relin_rescale(R, T, m * n, key, ctx, L, empty(ctx.mrr_scratch_bytes(L, m * n) // 8))
    dC = dev(C)
    he.ct_add(dC, dC, R, m * n, 2, ctx, L - 1)
    got = host(dC).reshape(m, n, 2, L, N)
    for (i, j) in ((0, 0), (13, 31), (31, 7)):
        t = oracle.tensor(A[i, 0], B[0, j], data)
        for l in range(1, k):
            t = oracle.add(t, oracle.tensor(A[i, l], B[l, j], data), data)
        ref = oracle.add(C[i, j], oracle.rescale(oracle.relin(t, evk, data, P, L), data, L), data[:L])
        assert np.array_equal(got[i, j], ref), (i, j)


def test_full_size_routines_sampled():
    """The routine set at N = 32K, 8 limbs, batches of 16 (the benchmark's
    configuration): two sampled ciphertexts per routine against the oracle."""
    N = 32768
    data, P = he.chain_primes(N, [60] + [50] * 7, 60)
    ctx = he.Context(N, data, P)
    r = Rng(170)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    key = he.RelinKey(ctx, evk)
    L, count = len(data) - 1, 16
    A, B = _cts(r, data, N, count), _cts(r, data, N, count)
    dA, dB = dev(A), dev(B)
    sc = empty(max(ctx.mrr_scratch_bytes(L, count), ctx.rotate_scratch_bytes(L, count)) // 8)
    out_l, out_r = empty(count, 2, L + 1, N), empty(count, 2, L, N)
    g = pow(5, 1, 2 * N)
    he.mul_relin(out_l, dA, dB, count, key, ctx, L, sc)
    ml = host(out_l)
    he.sqr_relin_rescale(out_r, dA, count, key, ctx, L, sc)
    sq = host(out_r)
    he.rotate(out_l, dA, count, g, key, ctx, L, sc)
    rt = host(out_l)
    for c in (0, 11):
        assert np.array_equal(ml[c], oracle.relin(oracle.tensor(A[c], B[c], data), evk, data, P, L)), c
        assert np.array_equal(sq[c], oracle.mul_relin_rescale(A[c], A[c], evk, data, P, L)), c
        assert np.array_equal(rt[c], oracle.rotate(A[c], g, evk, data, P, L)), c
