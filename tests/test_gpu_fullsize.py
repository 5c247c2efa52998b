"""GPU parity at the full sizes the benchmark runs, in its launch
configurations, on sampled outputs: the uneven batch (512 polynomials, N in
2^12..2^15, 1-16 limbs, seed 3) through the single mixed-degree launch and
the per-degree launches, and the element-wise 32 x 32 ciphertext matrix
product (1024 MulLinRS at N = 8192, 60/40/40 + 60-bit primes) as one call in
both evaluation shapes."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import empty, host  # noqa: E402


@pytest.mark.parametrize("per_degree", [False, True])
def test_uneven_batch_full_size(per_degree):
    pool = he.primes_generate(60, 1 << 16, 6) + he.primes_generate(55, 1 << 16, 5) + \
        he.primes_generate(50, 1 << 16, 5)
    degrees = [4096, 8192, 16384, 32768]
    tables = {N: he.NttTables(N, pool) for N in degrees}
    r = Rng(3)
    Ns = r.choice(degrees, 512)
    Ls = r.choice(list(range(1, 17)), 512)
    Fs = [min(int(f), 16 - L) for f, L in zip(r.choice(list(range(16)), 512), Ls)]
    xs = [r.uniform_limbs(pool[f:f + L], N) for N, L, f in zip(Ns, Ls, Fs)]
    ds = [torch.from_numpy(x.view(np.int64).copy()).cuda() for x in xs]
    entries = [(ds[i], tables[N], N, L, f) for i, (N, L, f) in enumerate(zip(Ns, Ls, Fs))]
    shapes = {N: he.ntt_shapes(N)[0][:2] for N in degrees} if per_degree else None
    plan = he.NttPlan(entries, shapes=shapes)
    assert plan.launches == (4 if per_degree else 1)
    plan.fwd()
    full = [i for i in range(512) if Ls[i] == 16][:2]
    sample = sorted({0, 1, 2, 128, 255, 384, 511} | {Ns.index(N) for N in degrees} | set(full))
    for i in sample:
        N, L, f = Ns[i], Ls[i], Fs[i]
        assert np.array_equal(host(ds[i]), oracle.ntt_fwd(xs[i], pool[f:f + L])), i
    plan.inv()
    torch.cuda.synchronize()
    for i in range(512):
        assert np.array_equal(ds[i].cpu().numpy().view(np.uint64), xs[i]), i


@pytest.mark.parametrize("log_e", [3, 4])
def test_elementwise_matrix_full_size(log_e):
    N, count, L = 8192, 1024, 2
    data, P = he.chain_primes(N, [60, 40, 40], 60)
    ctx = he.Context(N, data, P)
    ctx.set_eval_shape(log_e)
    r = Rng(4)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(3)])
    key = he.RelinKey(ctx, evk)
    A = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
    B = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
    out = empty(count, 2, L, N)
    he.mul_relin_rescale(out, torch.from_numpy(A.view(np.int64)).cuda(), torch.from_numpy(B.view(np.int64)).cuda(),
                         count, key, ctx, L, empty(ctx.mrr_scratch_bytes(L, count) // 8))
    got = host(out)
    for c in (0, 63, 64, 511, 1023):      # group boundaries of the expanded mod-up (64 ciphertexts)
        assert np.array_equal(got[c], oracle.mul_relin_rescale(A[c], B[c], evk, data, P, L)), c
