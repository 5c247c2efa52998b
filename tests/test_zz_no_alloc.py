"""The allocation-free mul-relin-rescale entry point, for callers that cannot
allocate device memory at call time (stream capture, allocator-free serving
paths, memory budgeted by another runtime). Called through the C ABI, its
output must equal the scratch-taking entry point's bit for bit, on two calls
in a row with different inputs (the built-in buffer keeps the first call's
contents, which must not leak into the second), and oversized requests must
be refused. The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402


def _setup():
    N = 4096
    data, P = he.chain_primes(N, [60, 50, 50, 50], 60)
    ctx = he.Context(N, data, P)
    r = Rng(99)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    return N, data, ctx, he.RelinKey(ctx, evk), r


def test_noalloc_matches_scratch_entry_point_twice():
    N, data, ctx, key, r = _setup()
    lib = he.load()
    stream = torch.cuda.current_stream().cuda_stream
    level, count = 3, 2
    for call in range(2):
        ca = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
        cb = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
        da, db = dev(ca), dev(cb)
        ref = empty(count, 2, level, N)
        scratch = empty(ctx.mrr_scratch_bytes(level, count) // 8)
        he.mul_relin_rescale(ref, da, db, count, key, ctx, level, scratch)
        got = empty(count, 2, level, N)
        got.fill_(-1)
        status = lib.he_mul_relin_rescale_noalloc(ctypes.c_void_p(got.data_ptr()), ctypes.c_void_p(da.data_ptr()),
                                                  ctypes.c_void_p(db.data_ptr()), count, key.handle, ctx.handle,
                                                  level, ctypes.c_void_p(stream))
        assert status == he.HE_OK, he.last_error()
        assert np.array_equal(host(got), host(ref)), f"call {call}"


def test_noalloc_rejects_oversized_requests():
    N, data, ctx, key, r = _setup()
    lib = he.load()
    level = 3
    per_pair = (3 * (level + 1) + 4) * N * 8
    too_many = he.NOALLOC_SCRATCH_BYTES // per_pair + 1
    d = empty(1)
    status = lib.he_mul_relin_rescale_noalloc(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                              ctypes.c_void_p(d.data_ptr()), too_many, key.handle, ctx.handle,
                                              level, None)
    assert status == he.HE_EINVAL
    assert "built-in" in he.last_error()


def test_noalloc_near_capacity_takes_the_fused_modup():
    """Five pairs at N = 2^14, level 6 (seven data primes) fill all but
    393 216 bytes of the built-in buffer, less than one ciphertext's expanded
    mod-up group, so the fused mod-up branch runs. Twice in a row, the output
    equals the scratch-taking entry point given a buffer of the same size."""
    N = 16384
    data, P = he.chain_primes(N, [60] + [50] * 6, 60)
    ctx = he.Context(N, data, P)
    r = Rng(98)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    key = he.RelinKey(ctx, evk)
    level, count = 6, 5
    need = (3 * (level + 1) + 4) * N * 8 * count
    group = (level + 2) * (level + 1) * N * 8
    assert need <= he.NOALLOC_SCRATCH_BYTES < need + group
    lib = he.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        ca = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
        cb = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
        da, db = dev(ca), dev(cb)
        ref = empty(count, 2, level, N)
        he.mul_relin_rescale(ref, da, db, count, key, ctx, level, empty(he.NOALLOC_SCRATCH_BYTES // 8))
        got = empty(count, 2, level, N)
        got.fill_(-1)
        status = lib.he_mul_relin_rescale_noalloc(ctypes.c_void_p(got.data_ptr()), ctypes.c_void_p(da.data_ptr()),
                                                  ctypes.c_void_p(db.data_ptr()), count, key.handle, ctx.handle,
                                                  level, ctypes.c_void_p(stream))
        assert status == he.HE_OK, he.last_error()
        assert np.array_equal(host(got), host(ref)), f"call {call}"
