"""GPU parity of the CKKS evaluation routines (Sec. II-A) through the C ABI:
Mul, Relin, RS and the fused MulLinRS, bit-exact against the CPU oracle on
the same seeded inputs, at several levels and batch sizes, plus decoded-slot
agreement on real encryptions."""
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
    "ckks16k": (16384, [60] + [50] * 6, 60),     # CKKS evaluation workload
    "matrix8k": (8192, [60, 40, 40], 60),        # element-wise matrix workload
    "small4k": (4096, [60, 50, 50, 50], 60),
}


def _relin_min_bytes(N, level):
    """The fused mod-up's minimum scratch, (3 n + 2) N words."""
    return (3 * (level + 1) + 2) * N * 8


def _mrr_min_bytes(N, level, count):
    """The fused mod-up's minimum MulLinRS scratch, (3 n + 4) N words a pair."""
    return (3 * (level + 1) + 4) * N * 8 * count


def _setup(name, seed):
    N, bits, pbits = CHAINS[name]
    data, P = he.chain_primes(N, bits, pbits)
    ctx = he.Context(N, data, P)
    r = Rng(seed)
    nd = len(data)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(nd)])
    key = he.RelinKey(ctx, evk)
    return N, data, P, ctx, evk, key, r


@pytest.mark.parametrize("name,level", [("ckks16k", 6), ("ckks16k", 3), ("matrix8k", 2), ("small4k", 0)])
def test_ct_mul(name, level):
    N, data, P, ctx, evk, key, r = _setup(name, 10 + level)
    qs = data[:level + 1]
    ca = np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
    cb = np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
    out = empty(3, level + 1, N)
    he.ct_mul(out, dev(ca), dev(cb), ctx, level)
    assert np.array_equal(host(out), oracle.tensor(ca, cb, qs))


@pytest.mark.parametrize("modup", ["expanded", "fused"])
@pytest.mark.parametrize("log_e", [4, 3])
@pytest.mark.parametrize("name,level", [("ckks16k", 6), ("ckks16k", 2), ("matrix8k", 2), ("small4k", 0),
                                        ("small4k", 3)])
def test_relin(name, level, log_e, modup):
    N, data, P, ctx, evk, key, r = _setup(name, 20 + level)
    ctx.set_eval_shape(log_e)
    qs = data[:level + 1]
    c3 = np.stack([r.uniform_limbs(qs, N) for _ in range(3)])
    out = empty(2, level + 1, N)
    nbytes = ctx.relin_scratch_bytes(level) if modup == "expanded" else _relin_min_bytes(N, level)
    scratch = empty(nbytes // 8)
    he.relin(out, dev(c3), key, ctx, level, scratch)
    assert np.array_equal(host(out), oracle.relin(c3, evk, data, P, level))


@pytest.mark.parametrize("log_e", [4, 3])
@pytest.mark.parametrize("name,level", [("ckks16k", 6), ("ckks16k", 1), ("matrix8k", 2), ("small4k", 3)])
def test_rescale(name, level, log_e):
    N, data, P, ctx, evk, key, r = _setup(name, 30 + level)
    ctx.set_eval_shape(log_e)
    qs = data[:level + 1]
    c = np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
    out = empty(2, level, N)
    scratch = empty(ctx.rescale_scratch_bytes(level) // 8)
    he.rescale(out, dev(c), ctx, level, scratch)
    assert np.array_equal(host(out), oracle.rescale(c, data, level))


@pytest.mark.parametrize("modup", ["expanded", "fused"])
@pytest.mark.parametrize("log_e", [4, 3])
@pytest.mark.parametrize("name,level,count", [("ckks16k", 6, 3), ("ckks16k", 2, 2), ("matrix8k", 2, 5),
                                              ("small4k", 1, 4), ("small4k", 3, 1)])
def test_mul_relin_rescale_batch(name, level, count, log_e, modup):
    N, data, P, ctx, evk, key, r = _setup(name, 40 + level + count)
    ctx.set_eval_shape(log_e)
    qs = data[:level + 1]
    ca = np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(count)])
    cb = np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(count)])
    out = empty(count, 2, level, N)
    nbytes = ctx.mrr_scratch_bytes(level, count) if modup == "expanded" else _mrr_min_bytes(N, level, count)
    assert _mrr_min_bytes(N, level, count) == ctx.mrr_scratch_bytes(level, count, 0)
    scratch = empty(nbytes // 8)
    he.mul_relin_rescale(out, dev(ca), dev(cb), count, key, ctx, level, scratch)
    got = host(out)
    for c in range(count):
        assert np.array_equal(got[c], oracle.mul_relin_rescale(ca[c], cb[c], evk, data, P, level)), c


@pytest.mark.parametrize("extra_polys", [11, 12, 36, 96])
def test_expanded_modup_groups(extra_polys):
    """11 pairs at level 2 (n = 3 limbs) with `extra_polys` x N words of
    scratch beyond the fused minimum: 11 holds no mod-up expansion
    ((n + 1) n = 12 per pair), so the fused mod-up runs; 12, 36 and 96 hold
    1, 3 and 8 (ragged last group). Same limbs as the oracle."""
    N, data, P, ctx, evk, key, r = _setup("small4k", 60 + extra_polys)
    level, count = 2, 11
    qs = data[:level + 1]
    ca = np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(count)])
    cb = np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)]) for _ in range(count)])
    out = empty(count, 2, level, N)
    nbytes = _mrr_min_bytes(N, level, count) + extra_polys * N * 8 + 8 * 5
    he.mul_relin_rescale(out, dev(ca), dev(cb), count, key, ctx, level, empty(nbytes // 8))
    got = host(out)
    for c in range(count):
        assert np.array_equal(got[c], oracle.mul_relin_rescale(ca[c], cb[c], evk, data, P, level)), c


def test_mul_relin_rescale_equals_composition():
    """The fused routine equals he_rescale(he_relin(he_ct_mul(a, b)))."""
    N, data, P, ctx, evk, key, r = _setup("small4k", 50)
    level = 3
    qs = data
    ca = np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
    cb = np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
    d3, d2, d1 = empty(3, 4, N), empty(2, 4, N), empty(2, 3, N)
    he.ct_mul(d3, dev(ca), dev(cb), ctx, level)
    he.relin(d2, d3, key, ctx, level, empty(ctx.relin_scratch_bytes(level) // 8))
    he.rescale(d1, d2, ctx, level, empty(ctx.rescale_scratch_bytes(level) // 8))
    fused = empty(1, 2, 3, N)
    he.mul_relin_rescale(fused, dev(ca[None]), dev(cb[None]), 1, key, ctx, level,
                         empty(ctx.mrr_scratch_bytes(level, 1) // 8))
    assert np.array_equal(host(fused)[0], host(d1))


@pytest.mark.parametrize("name,tol", [("matrix8k", 1e-5), ("ckks16k", 5e-5)])
def test_decoded_slots(name, tol):
    """Real encryptions: GPU MulLinRS limbs equal the oracle's bit for bit, and
    the decoded slots match the exact complex product (1e-5 relative at scale
    2^40; 5e-5 where 50-bit primes leave the output at scale 2^30)."""
    N, bits, pbits = CHAINS[name]
    data, P = oracle.chain_primes(N, bits, pbits)
    r = Rng(4)
    keys = ckks.keygen(N, data, P, r)
    scale = 2.0 ** 40
    za, zb = r.complex_slots(N // 2), r.complex_slots(N // 2)
    ca = ckks.encrypt(ckks.encode_real(za, N, scale), keys, r)
    cb = ckks.encrypt(ckks.encode_real(zb, N, scale), keys, r)
    L = len(data) - 1
    ctx = he.Context(N, data, P)
    key = he.RelinKey(ctx, keys.evk)
    out = empty(1, 2, L, N)
    he.mul_relin_rescale(out, dev(ca[None]), dev(cb[None]), 1, key, ctx, L, empty(ctx.mrr_scratch_bytes(L, 1) // 8))
    got = host(out)[0]
    ref = oracle.mul_relin_rescale(ca, cb, keys.evk, data, P, L)
    assert np.array_equal(got, ref)
    z = ckks.decrypt_decode(got, keys, scale * scale / data[L])
    exact = za * zb
    err = np.abs(z - exact).max() / max(1.0, np.abs(exact).max())
    assert err < tol, err


def test_full_ckks_workload_sampled():
    """64 ciphertext pairs at N = 16384 with seven data primes in one batched
    call, as the benchmark runs it; three pairs checked against the oracle."""
    N, data, P, ctx, evk, key, r = _setup("ckks16k", 2)
    L, count = 6, 64
    ca = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
    cb = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
    out = empty(count, 2, L, N)
    he.mul_relin_rescale(out, dev(ca), dev(cb), count, key, ctx, L, empty(ctx.mrr_scratch_bytes(L, count) // 8))
    got = host(out)
    for c in (0, 31, 63):
        assert np.array_equal(got[c], oracle.mul_relin_rescale(ca[c], cb[c], evk, data, P, L)), c


@pytest.mark.parametrize("count", [7, 8, 70])
def test_mul_relin_rescale_multiply_accumulate_forms(count):
    """The key multiply-accumulate of the expanded mod-up runs tiled (key
    pairs staged per position tile, groups of 8 or more ciphertexts) or per
    thread (smaller groups); 70 pairs make a tiled group of 64 followed by a
    per-thread group of 6. Every pair equals the one-pair call (per-thread
    form), and sampled pairs equal the oracle."""
    N, data, P, ctx, evk, key, r = _setup("matrix8k", 2)
    L = 2
    ca = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
    cb = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
    da, db = dev(ca), dev(cb)
    out = empty(count, 2, L, N)
    he.mul_relin_rescale(out, da, db, count, key, ctx, L, empty(ctx.mrr_scratch_bytes(L, count) // 8))
    got = host(out)
    one = empty(1, 2, L, N)
    s1 = empty(ctx.mrr_scratch_bytes(L, 1) // 8)
    for c in range(count):
        he.mul_relin_rescale(one, da[c:c + 1], db[c:c + 1], 1, key, ctx, L, s1)
        assert np.array_equal(got[c], host(one)[0]), c
    for c in {0, count // 2, count - 1}:
        assert np.array_equal(got[c], oracle.mul_relin_rescale(ca[c], cb[c], evk, data, P, L)), c
