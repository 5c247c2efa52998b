"""GPU parity of he_ntt_host, the pipelined transform of host-resident
batches (Sec. III asynchronous pipeline): forward, inverse and forward-then-
inverse against the oracle, with chunkings that leave a ragged last chunk,
pinned and pageable host memory, in-place use, and the argument checks."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, LIMBS, COUNT = 4096, 3, 37


@pytest.fixture(scope="module")
def setup():
    qs = he.primes_generate(60, 2 * N, 2) + he.primes_generate(50, 2 * N, 1)
    tables = he.NttTables(N, qs)
    r = Rng(0x4057)
    x = np.stack([r.uniform_limbs(qs, N) for _ in range(COUNT)])
    fwd = np.stack([oracle.ntt_fwd(x[c], qs) for c in range(COUNT)])
    return qs, tables, x, fwd


def _work(polys, extra_words=0):
    return torch.empty(polys * LIMBS * N + extra_words, dtype=torch.int64, device="cuda")


def _pinned(a):
    t = torch.from_numpy(a.reshape(-1).view(np.int64).copy()).pin_memory()
    return t


@pytest.mark.parametrize("work_polys,extra", [(1, 0), (5, 7), (12, 1), (64, 0)])
def test_forward_matches_oracle(setup, work_polys, extra):
    qs, tables, x, fwd = setup
    src = _pinned(x)
    dst = torch.zeros_like(src).pin_memory()
    he.ntt_host(src, dst, N, LIMBS, COUNT, tables, he.NTT_OP_FORWARD, _work(work_polys, extra))
    torch.cuda.synchronize()
    assert np.array_equal(dst.numpy().view(np.uint64).reshape(COUNT, LIMBS, N), fwd)
    assert np.array_equal(src.numpy().view(np.uint64).reshape(COUNT, LIMBS, N), x)


def test_inverse_matches_oracle_in_place(setup):
    qs, tables, x, fwd = setup
    buf = _pinned(fwd)
    he.ntt_host(buf, buf, N, LIMBS, COUNT, tables, he.NTT_OP_INVERSE, _work(8))
    torch.cuda.synchronize()
    assert np.array_equal(buf.numpy().view(np.uint64).reshape(COUNT, LIMBS, N), x)
    # the oracle's inverse agrees on one polynomial
    assert np.array_equal(oracle.ntt_inv(fwd[5], qs), x[5])


def test_round_trip_pageable_numpy(setup):
    qs, tables, x, fwd = setup
    src = np.ascontiguousarray(x)
    dst = np.zeros_like(src)
    he.ntt_host(src, dst, N, LIMBS, COUNT, tables, he.NTT_OP_FORWARD | he.NTT_OP_INVERSE, _work(6))
    torch.cuda.synchronize()
    assert np.array_equal(dst, x)


def test_ordered_on_caller_stream(setup):
    """Work queued on the caller's stream before the call is seen by it, and
    work queued after it sees its results."""
    qs, tables, x, fwd = setup
    s = torch.cuda.Stream()
    src = torch.zeros(COUNT * LIMBS * N, dtype=torch.int64).pin_memory()
    dst = torch.zeros_like(src).pin_memory()
    dev_in = torch.from_numpy(x.reshape(-1).view(np.int64).copy()).cuda()
    back = torch.zeros(COUNT * LIMBS * N, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        torch.cuda._sleep(20_000_000)   # keep the stream busy so that ordering matters
        src.copy_(dev_in, non_blocking=True)
        he.ntt_host(src, dst, N, LIMBS, COUNT, tables, he.NTT_OP_FORWARD, _work(4), stream=s)
        back.copy_(dst, non_blocking=True)
    s.synchronize()
    assert np.array_equal(back.cpu().numpy().view(np.uint64).reshape(COUNT, LIMBS, N), fwd)


def test_argument_checks(setup):
    qs, tables, x, fwd = setup
    src = np.ascontiguousarray(x)
    with pytest.raises(he.HeError) as e:
        he.ntt_host(src, src, N, LIMBS, COUNT, tables, 0, _work(4))
    assert e.value.status == he.HE_EINVAL
    with pytest.raises(he.HeError) as e:
        he.ntt_host(src, src, N, LIMBS, COUNT, tables, 4, _work(4))
    assert e.value.status == he.HE_EINVAL
    with pytest.raises(he.HeError) as e:   # scratch below one polynomial
        he.ntt_host(src, src, N, LIMBS, COUNT, tables, 1, _work(0, LIMBS * N - 2))
    assert e.value.status == he.HE_EINVAL
    big = np.zeros(2 * src.size, dtype=np.uint64)
    with pytest.raises(he.HeError) as e:   # partly overlapping host buffers
        he.ntt_host(big, big[8:], N, LIMBS, COUNT, tables, 1, _work(4))
    assert e.value.status == he.HE_EINVAL
    # nothing to do
    he.ntt_host(src, src, N, LIMBS, 0, tables, 1, _work(1))
