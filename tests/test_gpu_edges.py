"""Empty batches and rejected arguments across the whole boundary: every
batched entry point accepts count 0 and then writes nothing, and the host
checks turn bad levels, Galois elements, aliasing and short buffers into
errors before anything is launched (the output stays untouched)."""
import numpy as np
import pytest

from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402

N = 4096


@pytest.fixture(scope="module")
def env():
    data, P = he.chain_primes(N, [60, 50, 50], 60)
    ctx = he.Context(N, data, P)
    r = Rng(77)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(len(data))])
    key = he.RelinKey(ctx, evk)
    tables = he.NttTables(N, data)
    return data, P, ctx, key, tables, r


def _sentinel(*shape):
    t = empty(*shape)
    t.fill_(12345)
    return t


def _untouched(t):
    return bool((t == 12345).all().item())


def test_count_zero_everywhere(env):
    data, P, ctx, key, tables, r = env
    L = 2
    ct = dev(np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)])]))
    out = _sentinel(1, 2, L + 1, N)
    sc = empty(max(ctx.mrr_scratch_bytes(L, 1), ctx.rotate_scratch_bytes(L, 1)) // 8)
    he.ntt_fwd(out, N, 3, 0, tables)
    he.ntt_inv(out, N, 3, 0, tables)
    he.dyadic_mul(out, ct, ct, N, 3, 0, tables)
    he.negacyclic_mul(out, ct, ct, N, 3, 0, tables)
    he.mul_relin_rescale(out, ct, ct, 0, key, ctx, L, sc)
    he.sqr_relin_rescale(out, ct, 0, key, ctx, L, sc)
    he.mul_relin(out, ct, ct, 0, key, ctx, L, sc)
    he.ct_add(out, ct, ct, 0, 2, ctx, L)
    he.ct_automorph(out, ct, 0, 2, 5, ctx, L)
    he.rotate(out, ct, 0, 5, key, ctx, L, sc)
    he.mul_relin_rescale_batch([(out, ct, ct, 0, L)], key, ctx, sc)
    enc = he.Encoder(ctx)
    z = torch.zeros((1, N // 2), dtype=torch.complex128, device="cuda")
    he_sc = empty(enc.decode_scratch_bytes(L, 1) // 8)
    enc.encode(out, z, 0, 2.0 ** 40, L, he_sc)
    enc.decode(z, out, 0, 2.0 ** 40, L, he_sc)
    enc.crt_compose(torch.zeros((1, N), dtype=torch.float64, device="cuda"), out, 0, L)
    i8 = torch.zeros(N, dtype=torch.int8, device="cuda")
    he.encrypt(out, ct, dev(np.zeros((2, 3, N), dtype=np.uint64)), i8, i8, i8, 0, ctx, L, sc)
    torch.cuda.synchronize()
    assert _untouched(out)


def test_rejected_arguments_leave_outputs_untouched(env):
    data, P, ctx, key, tables, r = env
    L = 2
    ct = dev(np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)])]))
    out = _sentinel(1, 2, L + 1, N)
    sc = empty(ctx.mrr_scratch_bytes(L, 1) // 8)
    big = empty(1, 2, 4, N)
    cases = [
        lambda: he.mul_relin_rescale(out, big, big, 1, key, ctx, 3, sc),        # level beyond the chain
        lambda: he.mul_relin_rescale(out, ct, ct, 1, key, ctx, 0, sc),          # rescale needs level >= 1
        lambda: he.mul_relin_rescale(out, ct, ct, 1, key, ctx, L, sc[:64]),     # short scratch
        lambda: he.ct_automorph(out, ct, 1, 2, 4, ctx, L),                      # even Galois element
        lambda: he.ct_automorph(out, out, 1, 2, 5, ctx, L),                     # in place
        lambda: he.ntt_set_shape(N, 5, 3),                                      # shape not built
        lambda: he.ct_add(out, ct, ct, 1, 1, ctx, L),                           # components not 2 or 3
    ]
    for i, f in enumerate(cases):
        with pytest.raises(he.HeError):
            f()
        assert he.last_error(), i
    torch.cuda.synchronize()
    assert _untouched(out)


def test_binding_rejects_short_buffers(env):
    """The C ABI takes bare pointers; the binding checks each tensor against
    the words the call touches before anything reaches the library."""
    data, P, ctx, key, tables, r = env
    short = empty(N)
    sc = empty(ctx.mrr_scratch_bytes(2, 1) // 8)
    with pytest.raises(ValueError):
        he.ntt_fwd(short, N, 3, 1, tables)
    with pytest.raises(ValueError):
        he.mul_relin_rescale(short, short, short, 1, key, ctx, 2, sc)
    with pytest.raises(ValueError):
        he.negacyclic_mul(short, short, short, N, 2, 1, tables)
    with pytest.raises(ValueError):
        he.encrypt(short, short, short, torch.zeros(N, dtype=torch.int8, device="cuda"),
                   torch.zeros(N, dtype=torch.int8, device="cuda"), torch.zeros(N, dtype=torch.int8, device="cuda"),
                   1, ctx, 2, sc)


def test_buffers_must_be_32_byte_aligned(env):
    """Runs of four consecutive words move with 256-bit accesses, so the
    boundary requires 32-byte aligned device buffers: a buffer 16 bytes off
    that is refused before anything is launched, and nothing is written."""
    data, P, ctx, key, tables, r = env
    L = 2
    flat = _sentinel(L * N + 2)
    off = flat[2:]                                    # 16 bytes past an aligned start
    assert off.data_ptr() % 32 == 16
    ct = dev(np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)])]))
    ct_flat = _sentinel(2 * (L + 1) * N + 2)
    ct_off = ct_flat[2:].view(1, 2, L + 1, N)
    out_flat = _sentinel(2 * L * N + 2)
    out_off = out_flat[2:].view(1, 2, L, N)
    sc = empty(ctx.mrr_scratch_bytes(L, 1) // 8)
    sc_off = empty(ctx.mrr_scratch_bytes(L, 1) // 8 + 2)[2:]
    cases = [
        lambda: he.ntt_fwd(off, N, L, 1, tables),
        lambda: he.ntt_inv(off, N, L, 1, tables),
        lambda: he.dyadic_mul(empty(L * N), off, off, N, L, 1, tables),
        lambda: he.mul_relin_rescale(out_off, ct, ct, 1, key, ctx, L, sc),
        lambda: he.mul_relin_rescale(empty(1, 2, L, N), ct_off, ct, 1, key, ctx, L, sc),
        lambda: he.mul_relin_rescale(empty(1, 2, L, N), ct, ct, 1, key, ctx, L, sc_off),
    ]
    for i, f in enumerate(cases):
        with pytest.raises(he.HeError, match="32-byte"):
            f()
    torch.cuda.synchronize()
    assert _untouched(flat) and _untouched(ct_flat) and _untouched(out_flat)
